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
// holds S A-slice tiles and S Omega-slice tiles.  The slicers write the digits
// in exactly that shared-memory image, tile after tile, so a stage's A tiles
// are one contiguous block in memory and arrive by one bulk copy (rather than
// a tensor copy of 64-byte rows per tile).  Every CTA loads its own tiles:
// nothing is multicast between CTAs.  A K-split over CTAs balances
// the waves; partial sums are reduced in a fixed order, so results are
// deterministic.  Row probes (rows l.. of Omega) are sliced and multiplied
// like the test matrix's rows and reduced into X instead of Y.
#include <climits>

#include "rid_internal.cuh"
#include "rid_tc.cuh"
#include "rid_tc_digits.cuh"

using namespace rid_tc;

namespace {

struct TcState {
  int S;
  int row0, nrows;        // the rows of Omega this state multiplies
  int nstages;            // pipeline stages that fit in shared memory
  uint32_t stage_smem, o_off, o_tile_smem;   // o_tile_smem: tile_w (pairs: tile_w / 2) rows x 64 bytes
  int dyn_smem;           // dynamic shared memory of the product kernel
  int so;                 // Omega digits used: S, or bits / 8 for a rounded Omega
  int64_t KP;             // padded reduction length (multiple of TC_KC)
  int64_t nst;            // K stages: KP / TC_KS
  int NC;                 // chunks
  int l2;                 // 2l rows of Omega'
  int ntiles;             // N-tiles of tile_w <= 128 rows (balanced: the cluster runs at the widest)
  int tile_w;             // rows of Omega' per N-tile, a multiple of 16
  int nblocks;            // column blocks of 128
  int ksplit;             // K-splits
  int chunks_per_split;
  bool pair;              // CTA pairs (M = 256) rather than single CTAs
  int cx;                 // single CTAs: N-tiles per cluster
  uint16_t* om_slices;    // tiles [N-tile][K stage][S][tile_w x TC_KS] bf16 (see omega_slice_kernel)
  int* om_exp;            // [l2]
  uint16_t* a_slices;     // tiles [column block of the panel][K stage][S][128 x TC_KS] bf16 (see a_slice_kernel)
  int panel_blocks;       // column blocks of one panel: the digit tiles hold one panel at a time
  int* a_exp;             // [n][NC]
  int* a_exp_max;         // [n]
  float2* partial;        // [ksplit][n][l2p]: (hi, lo) of each running sum
  int l2p;
  int* err;               // device error word
};

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

// Digits of Omega' rows: row 2i = (Re w_r, -Im w_r), row 2i+1 = (Im w_r, Re w_r),
// written as the product kernel's Omega tiles in the swizzled image of
// tile_offset: [N-tile][K stage][digit] tiles of tile_w rows x TC_KS bf16 for
// single CTAs; for CTA pairs [N-tile][K stage][half][digit] tiles of
// tile_w / 2 rows, half 0 holding the tile's rows below n / 2 and half 1 the
// rest (n = tile_mma_n).  Rows past 2l stay as the caller zeroed them.
__global__ void omega_slice_kernel(const double2* __restrict__ om, int64_t ldo, int64_t m, int l, int64_t KP,
                                   int tile_w, bool pair, const int* __restrict__ om_exp,
                                   uint16_t* __restrict__ tiles) {
  const int64_t per_row = KP / 2;      // complex positions per row, incl. padding
  const int64_t total = (int64_t)l * per_row;
  const int64_t nst = KP / TC_KS;
  const int H = pair ? 2 : 1;
  const int64_t tile_elems = (int64_t)(tile_w / H) * TC_KS;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / per_row);
    const int64_t r = e - (int64_t)i * per_row;
    const double2 w = r < m ? om[i * ldo + r] : make_double2(0.0, 0.0);
    const int ex = om_exp[2 * i];
    uint16_t re[TC_S], nim[TC_S], im[TC_S];
    digits_of(w.x, ex, re);
    digits_of(-w.y, ex, nim);
    digits_of(w.y, ex, im);
    const int64_t st = 2 * r / TC_KS;               // K stage of reals 2r, 2r + 1
    const int k = (int)(2 * r - st * TC_KS);        // their position in the stage (even)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = 2 * i + h, nt = row / tile_w, rr = row - nt * tile_w;
      int hh = 0, r = rr;
      if (pair) {
        const int half = tile_mma_n(tile_w, 2 * l, nt, true) / 2;
        hh = rr >= half ? 1 : 0;
        r = rr - hh * half;
      }
      uint16_t* dst = tiles + (((int64_t)nt * nst + st) * H + hh) * TC_S * tile_elems + tile_offset(r, k) / 2;
      for (int s = 0; s < TC_S; ++s)
        *(uint32_t*)(dst + s * tile_elems) =
            h == 0 ? (uint32_t)re[s] | ((uint32_t)nim[s] << 16) : (uint32_t)im[s] | ((uint32_t)re[s] << 16);
    }
  }
}

// ---- A' slices (every call) -------------------------------------------------------
// A block of 8 warps takes 8 consecutive columns j0 .. j0+7 of one chunk c;
// warp w slices column j0 + w: 128 complex rows = 256 real values, a lane 4
// consecutive complex rows, i.e. one 16-byte chunk of one K stage's tile row.
// Column j is row j % 128 of the tiles of column block j / 128:
// [column block][K stage][digit] tiles of 128 rows x TC_KS bf16 in the
// swizzled image of tile_offset.  The 8 rows of the block form one 512-byte
// swizzle atom in each of the chunk's 8 stages x S digits: they are gathered
// in shared memory and stored atom by atom, 512 contiguous bytes per warp
// store; the next task's loads are issued before those stores.  Columns
// n .. n_pad - 1 (the last block's padding) get zero digits.
template <typename TA>
__device__ __forceinline__ void slice_load(const TA* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                                           int64_t groups, int64_t t, int warp, int lane, double2 (&x)[4]) {
  const int c = (int)(t / groups);
  const int64_t j = (t - (int64_t)c * groups) * 8 + warp;
  const int64_t r0 = (int64_t)c * 128 + 4 * lane;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (j < n && r0 + u < m) {
      const TA v = __ldg(A + j * lda + r0 + u);
      x[u] = make_double2((double)v.x, (double)v.y);     // exact for complex64 input
    } else {
      x[u] = make_double2(0.0, 0.0);
    }
  }
}

template <typename TA>
__global__ void __launch_bounds__(256) a_slice_kernel(const TA* __restrict__ A, int64_t lda, int64_t m,
                                                      int64_t n, int64_t n_pad, int NC,
                                                      uint16_t* __restrict__ tiles, int* __restrict__ a_exp,
                                                      int* __restrict__ a_exp_max) {
  // A, tiles, a_exp and a_exp_max start at the first column of the range
  // (n columns, a multiple of 128 from the matrix's first column)
  __shared__ uint4 atoms[TC_SPC * TC_S][8][4];         // [stage x digit][row][16-byte chunk]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t groups = n_pad / 8;                  // 8-column groups per chunk
  const int64_t tasks = groups * NC;
  const int64_t nst = (int64_t)NC * TC_SPC;
  double2 x[4];
  int64_t t = blockIdx.x;
  if (t < tasks) slice_load(A, lda, m, n, groups, t, warp, lane, x);
  for (; t < tasks; t += gridDim.x) {
    const int c = (int)(t / groups);
    const int64_t j0 = (t - (int64_t)c * groups) * 8;
    const int64_t j = j0 + warp;
    int e = TC_EXP_ZERO;
#pragma unroll
    for (int u = 0; u < 4; ++u) e = max(e, max(exp_of(x[u].x), exp_of(x[u].y)));
    e = __reduce_max_sync(0xffffffffu, e);
    uint32_t w[4][TC_S];
#pragma unroll
    for (int u = 0; u < 4; ++u) digit_words(x[u], e, w[u]);
    // reals 2 r0 .. 2 r0 + 7: stage lane / 4 of the chunk, elements 8 (lane % 4) .. + 7
    // of tile row j % 128 (row `warp` of its atom; the swizzle depends on the row's bits 1-2)
    const int row = (int)(j & 127);
    const int pc = (lane & 3) ^ ((row >> 1) & 3);
#pragma unroll
    for (int s = 0; s < TC_S; ++s)
      atoms[(lane >> 2) * TC_S + s][warp][pc] = make_uint4(w[0][s], w[1][s], w[2][s], w[3][s]);
    if (lane == 0 && j < n) {
      a_exp[j * NC + c] = e;
      atomicMax(a_exp_max + j, e);
    }
    __syncthreads();
    if (t + gridDim.x < tasks) slice_load(A, lda, m, n, groups, t + gridDim.x, warp, lane, x);
    uint16_t* dst = tiles + ((j0 >> 7) * nst + (int64_t)c * TC_SPC) * TC_S * TC_TILE_ELEMS + (j0 & 127) * TC_KS;
    for (int a = warp; a < TC_SPC * TC_S; a += 8)       // atom a = (stage a / S, digit a % S)
      ((uint4*)(dst + (int64_t)a * TC_TILE_ELEMS))[lane] = (&atoms[a][0][0])[lane];
    __syncthreads();
  }
}

// ---- the tensor-core product ----------------------------------------------------------
// Two forms of one kernel.  Single CTAs (PAIR = false): M = 128 columns of A
// per CTA, each CTA loading its own A and Omega tiles (clusters of 1).  CTA
// pairs (PAIR = true): one tcgen05 MMA of M = 256
// (cta_group::2) covers two column blocks; each CTA of the pair holds its
// block's A tiles and half of the N-tile's Omega rows, and the tensor cores of
// the pair read each half once.  That halves the Omega bytes per CTA (shared
// memory traffic bounds the single form at N = 112: the MMA's operand reads
// plus the TMA fill exceed what the SM's shared memory delivers).
struct TcArgs {
  int n, l2, l2p, NC, chunks_per_split, ntiles, tile_w;
  uint32_t stage_bytes;   // bytes landing in one CTA's stage: S A tiles + so Omega tiles
  int so;                 // Omega digits that can be non-zero (S, or fewer for a rounded Omega)
  int nstages;            // pipeline stages
  uint32_t stage_smem;    // shared memory of one stage (1024-byte multiple)
  uint32_t o_off;         // offset of the Omega tiles in a stage
  uint32_t o_tile_smem;   // one Omega tile: tile_w rows (single) or tile_w / 2 rows (pairs) x 64 bytes
  int cx;                 // single CTAs: N-tiles per cluster (they share A tiles)
  int jb0;                // first column block of the launch (a column range of the sketch)
  int tile_jb0;           // the column block whose digit tiles start a_tiles
  int64_t j_end;          // columns below this have results in the launch
  int64_t nst;            // K stages per column block / N-tile
  const uint16_t* a_tiles;
  const uint16_t* om_tiles;
  const int* a_exp;
  const int* a_exp_max;
  float2* partial;
  int* err;
};

template <bool PAIR>
__global__ void __launch_bounds__(TC_THREADS, 1) sketch_tc_kernel(TcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full_bar[TC_MAX_STAGES], empty_bar[TC_MAX_STAGES], peer_full[TC_MAX_STAGES];
  __shared__ uint64_t acc_full[TC_G], acc_empty[TC_G], mma_done;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // Single: grid (N-tiles, column blocks, K-splits), clusters of cx N-tiles.
  // Pairs: grid (2 x N-tiles, column-block pairs, K-splits), clusters of the
  // two CTAs of one N-tile (member 0 leads: it issues the MMAs).
  const int member = PAIR ? (int)(blockIdx.x & 1) : 0;
  const int nb = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int jb = a.jb0 + (PAIR ? 2 * (int)blockIdx.y + member : (int)blockIdx.y);
  const int ks = blockIdx.z;
  const uint32_t my_rank = PAIR ? (uint32_t)member : (uint32_t)(nb % a.cx);
  const uint16_t all_mask = PAIR ? (uint16_t)3 : (uint16_t)((1u << a.cx) - 1u);
  const bool leader = member == 0;
  const int c_begin = ks * a.chunks_per_split;
  const int c_end = min(a.NC, c_begin + a.chunks_per_split);
  const int nchunks = max(0, c_end - c_begin);
  const int row0 = nb * a.tile_w;
  const int n_tile = min(a.tile_w, a.l2 - row0);
  const int n_mma = tile_mma_n(a.tile_w, a.l2, nb, PAIR);

  if (warp == 13) {
    if (PAIR) tmem_alloc_pair(&tmem_slot, 512);
    else tmem_alloc(&tmem_slot, 512);
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < a.nstages; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&empty_bar[i], PAIR ? 1 : a.cx);   // released by the MMA issuer(s) of the cluster
      mbar_init(&peer_full[i], 1);
    }
    for (int g = 0; g < TC_G; ++g) {
      mbar_init(&acc_full[g], 1);
      mbar_init(&acc_empty[g], PAIR ? 2 * TC_FLUSH_WARPS : TC_FLUSH_WARPS);
    }
    mbar_init(&mma_done, 1);
    fence_barrier_init();
    s_abort = cluster_rank() != my_rank ? 1 : 0;      // grid and cluster layout disagree
    if (s_abort) atomicCAS(a.err, 0, 1);
  }
  tc_fence_before();
  cluster_sync();          // a pair's barriers initialised before the other CTA signals them
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
      // This CTA's A tiles of each stage (a cluster of one, or its half of a
      // pair), then its Omega tiles; each is one contiguous block of the tile
      // arrays.
      const int s0 = 0, s1 = TC_S;
      const int o_elems = (int)(a.o_tile_smem / 2);
      const int64_t st0 = (int64_t)c_begin * TC_SPC;            // first K stage of this split
      const uint16_t* a_src = a.a_tiles + (((int64_t)(jb - a.tile_jb0) * a.nst + st0) * TC_S + s0) * TC_TILE_ELEMS;
      const uint16_t* o_src = PAIR ? a.om_tiles + ((nb * a.nst + st0) * 2 + member) * TC_S * o_elems
                                   : a.om_tiles + (nb * a.nst + st0) * TC_S * o_elems;
      const int64_t o_stride = (PAIR ? 2 : 1) * TC_S * (int64_t)o_elems;
      const uint32_t a_bytes = (uint32_t)(s1 - s0) * TC_TILE_BYTES, o_bytes = (uint32_t)a.so * a.o_tile_smem;
      const int iters = nchunks * TC_SPC;
      int it = 0, slot = 0, round = 0;
      for (; it < iters && !s_abort; ++it) {
        if (round > 0 && !mbar_wait(&empty_bar[slot], (round - 1) & 1, TC_WAIT_BUDGET)) {
          fail(11);
          break;
        }
        // the stage's 2S tiles arrive here whoever issued them
        mbar_arrive_expect_tx(&full_bar[slot], a.stage_bytes);
        if (a_bytes) {
          bulk_load(a_tile(slot, s0), a_src, a_bytes, &full_bar[slot]);
        }
        bulk_load(o_tile(slot, 0), o_src, o_bytes, &full_bar[slot]);
        a_src += TC_S * TC_TILE_ELEMS;        // next K stage
        o_src += o_stride;
        if (++slot == NS) {
          slot = 0;
          ++round;
        }
      }
      // tail: before the CTA may exit, every slot must have been released by
      // every MMA issuer of the cluster (their commits arrive here), or, after
      // an error, every load issued into this CTA must have landed
      for (int k = max(0, it - NS); k < it; ++k) {
        const bool ok = s_abort ? mbar_wait(&full_bar[k % NS], (k / NS) & 1, TC_WAIT_BUDGET)
                                : mbar_wait(&empty_bar[k % NS], (k / NS) & 1, TC_WAIT_BUDGET);
        if (!ok) fail(12);
      }
    } else if (warp == 13 && leader) {
      // ---------------- MMA issuer (the whole warp; one elected lane issues) ----------------
      const uint32_t idesc = idesc_bf16_f32(PAIR ? 256 : 128, n_mma);
      const int stages_per_chunk = TC_SPC;
      // descriptor start addresses are in 16-byte units (low 14 bits): a tile
      // offset within the CTA's shared memory adds without carry
      const uint64_t o_step = a.o_tile_smem >> 4;
      int slot = 0, round = 0;
      for (int cl = 0; cl < nchunks && !s_abort; ++cl) {
        for (int b = 0; b < stages_per_chunk && !s_abort; ++b) {
          // this CTA's tiles, and for a pair the other CTA's (relayed)
          if (!__all_sync(0xffffffffu, mbar_wait(&full_bar[slot], round & 1, TC_WAIT_BUDGET) &&
                                        (!PAIR || mbar_wait_cluster(&peer_full[slot], round & 1, TC_WAIT_BUDGET)))) {
            if (lane == 0) fail(21);
            break;
          }
          tc_fence_after();
          const uint64_t da0 = tile_desc(a_tile(slot, 0)), db0 = tile_desc(o_tile(slot, 0));
          bool ok = true;
          switch (a.so) {      // the Omega digit count picks a fully unrolled issue sequence
#define RID_MMA_STAGE(SO) \
            case SO: ok = mma_stage<SO, PAIR>(tmem, da0, db0, o_step, idesc, b, cl, stages_per_chunk, acc_empty, acc_full); break;
            RID_MMA_STAGE(1) RID_MMA_STAGE(2) RID_MMA_STAGE(3) RID_MMA_STAGE(4) RID_MMA_STAGE(5) RID_MMA_STAGE(6)
            RID_MMA_STAGE(7)
#undef RID_MMA_STAGE
            default: ok = false;
          }
          if (!ok) {
            if (lane == 0) fail(22);
            break;
          }
          if (PAIR) mma_commit_pair_multicast_w(&empty_bar[slot], all_mask);
          else mma_commit_w(&empty_bar[slot]);
          if (++slot == NS) {
            slot = 0;
            ++round;
          }
        }
      }
      if (PAIR) mma_commit_pair_multicast_w(&mma_done, all_mask);
      else mma_commit_w(&mma_done);
    } else if (PAIR && warp == 13 && lane == 0) {
      // ---------------- relay (odd CTA of a pair) ----------------
      // the leader's MMAs read this CTA's tiles: tell it when each stage has landed
      const int iters = nchunks * TC_SPC;
      int slot = 0, round = 0;
      for (int it = 0; it < iters && !s_abort; ++it) {
        if (!mbar_wait(&full_bar[slot], round & 1, TC_WAIT_BUDGET)) {
          fail(23);
          break;
        }
        mbar_arrive_remote(&peer_full[slot], 0);
        if (++slot == NS) {
          slot = 0;
          ++round;
        }
      }
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
    const bool j_ok = j < a.j_end;
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
              if (lane == 0) {
                if (leader) mbar_arrive(&acc_empty[g]);
                else mbar_arrive_remote(&acc_empty[g], 0);   // the pair's MMAs are the leader's
              }
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
    if (PAIR) tmem_dealloc_pair(tmem, 512);
    else tmem_dealloc(tmem, 512);
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
    const float4* p = (const float4*)(partial + j * l2p + 2 * i);   // (hi, lo) of rows 2i and 2i+1
    const int64_t split_stride = n * l2p / 2;                       // float4 units
    // the splits in order; their loads batched ahead of the additions
    for (int s0 = 0; s0 < ksplit; s0 += 8) {
      float4 q[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (s0 + u < ksplit) q[u] = __ldcs(p + (int64_t)(s0 + u) * split_stride);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (s0 + u < ksplit) {
          re += (double)q[u].x + (double)q[u].y;
          im += (double)q[u].z + (double)q[u].w;
        }
    }
    const int ea = a_exp_max[j];
    const double2 v = make_double2(ea == TC_EXP_ZERO ? 0.0 : ldexp(re, om_exp[2 * i] + ea - 16),
                                   ea == TC_EXP_ZERO ? 0.0 : ldexp(im, om_exp[2 * i + 1] + ea - 16));
    if (i < ly) Y[i + j * ldy] = v;
    else X[(i - ly) + j * ldx] = v;
  }
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

int rid_tc_choose_ksplit(int units, int NC, int slots) { return choose_ksplit(units, NC, slots); }

cudaError_t rid_tc_cut_omega(const double2* om, int64_t ldo, int64_t m, int nrows, int64_t KP, int tile_w, bool pair,
                             int* om_exp, uint16_t* tiles, int num_sms, cudaStream_t stream) {
  omega_exp_kernel<<<nrows, 256, 0, stream>>>(om, ldo, m, om_exp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int64_t blocks = ((int64_t)nrows * (KP / 2) + 255) / 256;
  if (blocks > (int64_t)num_sms * 32) blocks = (int64_t)num_sms * 32;
  omega_slice_kernel<<<(unsigned)blocks, 256, 0, stream>>>(om, ldo, m, nrows, KP, tile_w, pair, om_exp, tiles);
  return cudaGetLastError();
}

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
// tiles, the A digit tile buffer, exponents and partial sums.  dry_run: only
// the device bytes.
rid_status tc_setup(rid_plan_s* p, int dry_run, int row0, int nrows, TcState** out,
                    size_t* bytes_out) {
  *out = nullptr;
  TcState* st = (TcState*)calloc(1, sizeof(TcState));
  if (!st) return RID_ENOMEM;
  st->S = TC_S;
  st->row0 = row0;
  st->nrows = nrows;
  // a rounded Omega holds omega_bits / 8 digits relative to its row exponent,
  // the same exponent omega_exp_kernel takes, so the others are exactly zero
  st->so = p->omega_bits > 0 ? (p->omega_bits + 7) / 8 : TC_S;
  st->NC = (int)((2 * p->m + TC_KC - 1) / TC_KC);
  st->KP = (int64_t)st->NC * TC_KC;
  st->nst = st->KP / TC_KS;
  st->l2 = 2 * nrows;
  st->ntiles = (st->l2 + 127) / 128;
  st->tile_w = ((st->l2 + st->ntiles - 1) / st->ntiles + 15) / 16 * 16;
  st->nblocks = (int)((p->n + 127) / 128);
  // CTA pairs for 16 or more column blocks (an odd count multiplies one
  // block of zeros, so small problems lose more than the pairs gain; a batch
  // of 64..1024-column IDs ran 5 % faster on single CTAs) with at least 32
  // rows to split between the pair (its MMA takes N >= 32; a narrower tile,
  // e.g. the row probes alone, runs faster on single CTAs than padded)
  st->pair = st->nblocks >= 16 && st->l2 >= 32;
  if (st->pair && st->tile_w < 32) st->tile_w = 32;
  st->l2p = st->ntiles * st->tile_w;
  // Column panels: the digit tiles of A take 7/4 of A's bytes, so a matrix of
  // more than 32 column blocks is sliced and multiplied in at most 4 panels
  // (even block counts, so CTA pairs never straddle two panels): the plan's
  // digit tiles stay below half of A's bytes.
  {
    const int np = st->nblocks > 32 ? 4 : 1;
    int pb = (st->nblocks + np - 1) / np;
    if (st->pair) pb = (pb + 1) & ~1;
    st->panel_blocks = pb;
  }
  if (st->ntiles > 8) {
    free(st);
    return RID_EUNSUPPORTED;
  }
  // Stage layout: S A tiles, then so Omega tiles of tile_w rows (pairs:
  // tile_w / 2), a multiple of 8 rows, so every tile starts where its
  // 512-byte swizzle pattern does; as many stages as shared memory holds.
  st->o_tile_smem = (uint32_t)((st->pair ? st->tile_w / 2 : st->tile_w) * TC_KS * 2);
  st->o_off = (uint32_t)(TC_S * TC_TILE_BYTES);
  st->stage_smem = (st->o_off + (uint32_t)st->so * st->o_tile_smem + 1023) / 1024 * 1024;
  st->nstages = (int)((TC_SMEM_LIMIT - 2048 - 1024) / st->stage_smem);
  if (st->nstages > TC_MAX_STAGES) st->nstages = TC_MAX_STAGES;
  if (st->nstages < 2) {
    free(st);
    return RID_EUNSUPPORTED;
  }
  st->dyn_smem = (int)(st->nstages * st->stage_smem + 1024);
  // Single CTAs: clusters of one (each CTA loads its own A tiles; sharing
  // them across the N-tiles of a column block by multicast bought about 1 %).
  // Pairs: a cluster is the pair.
  st->cx = st->pair ? 2 : 1;
  // clusters per K-split of one panel
  const int units = st->pair ? st->ntiles * (st->panel_blocks / 2) : st->ntiles * st->panel_blocks;
  {
    // how many clusters of this shape are resident at once
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(st->pair ? 2 * st->ntiles : st->ntiles, st->pair ? (st->nblocks + 1) / 2 : st->nblocks, 1);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = st->dyn_smem;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = st->cx;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    const void* fn = st->pair ? (const void*)sketch_tc_kernel<true> : (const void*)sketch_tc_kernel<false>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_DYN_SMEM_MAX);
    if (cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) != cudaSuccess || clusters < 1) {
      cudaGetLastError();
      clusters = p->num_sms / st->cx;
    }
    st->ksplit = choose_ksplit(units, st->NC, clusters > 0 ? clusters : 1);
  }
  st->chunks_per_split = (st->NC + st->ksplit - 1) / st->ksplit;
  st->ksplit = (st->NC + st->chunks_per_split - 1) / st->chunks_per_split;

  const size_t om_bytes = (size_t)TC_S * st->l2p * st->KP * 2;           // N-tiles padded to tile_w rows
  const size_t block_bytes = (size_t)TC_S * 128 * st->KP * 2;            // one column block's tiles
  const size_t a_bytes = block_bytes * st->panel_blocks;
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

  cudaError_t e = cudaMemsetAsync(st->err, 0, 4, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(st->om_slices, 0, om_bytes, p->stream);   // padding rows
  if (e == cudaSuccess)
    e = rid_tc_cut_omega(p->omega + (int64_t)row0 * p->ldo, p->ldo, p->m, nrows, st->KP, st->tile_w, st->pair,
                         st->om_exp, st->om_slices, p->num_sms, p->stream);
  const void* fn = st->pair ? (const void*)sketch_tc_kernel<true> : (const void*)sketch_tc_kernel<false>;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_DYN_SMEM_MAX);
  if (e == cudaSuccess) {
    // setmaxnreg moves registers between warpgroups inside the launch
    // allocation; it is only safe if the kernel launches with exactly the
    // 128 registers per thread the split adds up to.
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fn);
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
  const rid_status s = tc_setup(p, dry_run, 0, p->ls, &st, &bytes);   // the test matrix and the row probes
  if (s != RID_OK) return s;
  p->tc_bytes = bytes;
  if (!dry_run) {
    p->tc_state = st;
    // a whole-matrix sketch: slicing and product per column panel, then the reduction
    p->tc_sketch_launches = 2 * ((st->nblocks + st->panel_blocks - 1) / st->panel_blocks) + 1;
  }
  return RID_OK;
}

void rid_tc_plan_free_fp64(rid_plan_s* p) {
  tc_free_state(p, (TcState*)p->tc_state);
  p->tc_state = nullptr;
  p->tc_bytes = 0;
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
  // the range's column blocks, a panel of at most panel_blocks at a time: its
  // digits are cut into the plan's tiles, then multiplied
  const int jb_begin = (int)(col0 / 128), jb_end = (int)((col0 + ncols + 127) / 128);
  const int npanels = (jb_end - jb_begin + st->panel_blocks - 1) / st->panel_blocks;
  if (timing) {
    p->ev_panels = npanels <= RID_MAX_PANELS ? npanels : 0;
    cudaEventRecord(p->ev[0], p->stream);
  }
  // 0x80808080 is below every exponent: the running maximum starts there
  cudaError_t e = cudaMemsetAsync(st->a_exp_max + col0, 0x80, (size_t)ncols * 4, p->stream);
  if (e != cudaSuccess) return e;
  for (int pi = 0; pi < npanels; ++pi) {
    const int jb0 = jb_begin + pi * st->panel_blocks;
    const int nblocks = jb_end - jb0 < st->panel_blocks ? jb_end - jb0 : st->panel_blocks;
    const int64_t c0 = (int64_t)jb0 * 128;                      // the panel's first column
    const int64_t pcols = (col0 + ncols < c0 + (int64_t)nblocks * 128 ? col0 + ncols : c0 + (int64_t)nblocks * 128) - c0;
    {
      // a CTA pair's partner of an odd last block gets zero digits
      const int64_t n_pad = st->pair ? (pcols + 255) / 256 * 256 : (pcols + 127) / 128 * 128;
      int64_t blocks = n_pad / 8 * (int64_t)st->NC;          // a block per 8 columns of one chunk
      if (blocks > (int64_t)p->num_sms * 16) blocks = (int64_t)p->num_sms * 16;
      a_slice_kernel<double2><<<(unsigned)blocks, 256, 0, p->stream>>>(
            (const double2*)A_ + c0 * lda, lda, p->m, pcols, n_pad, st->NC, st->a_slices, st->a_exp + c0 * st->NC,
            st->a_exp_max + c0);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (timing && pi < RID_MAX_PANELS && p->ev_panels) cudaEventRecord(p->ev[1 + 2 * pi], p->stream);
    TcArgs args{(int)p->n, st->l2, st->l2p, st->NC, st->chunks_per_split, st->ntiles, st->tile_w,
                (uint32_t)(TC_S * TC_TILE_BYTES) + (uint32_t)st->so * st->o_tile_smem, st->so, st->nstages,
                st->stage_smem, st->o_off, st->o_tile_smem, st->cx, jb0, jb0, c0 + pcols, st->nst, st->a_slices,
                st->om_slices, st->a_exp, st->a_exp_max, st->partial, st->err};
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = st->pair ? dim3((unsigned)(2 * st->ntiles), (unsigned)((nblocks + 1) / 2), (unsigned)st->ksplit)
                           : dim3((unsigned)st->ntiles, (unsigned)nblocks, (unsigned)st->ksplit);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = st->dyn_smem;
    cfg.stream = p->stream;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = st->cx;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = st->pair ? cudaLaunchKernelEx(&cfg, sketch_tc_kernel<true>, args)
                 : cudaLaunchKernelEx(&cfg, sketch_tc_kernel<false>, args);
    if (e != cudaSuccess) return e;
    if (timing && pi < RID_MAX_PANELS && p->ev_panels) cudaEventRecord(p->ev[2 + 2 * pi], p->stream);
  }
  if (timing && !p->ev_panels) {        // more panels than timed: the whole sketch counts as its first pass
    p->ev_panels = 1;
    cudaEventRecord(p->ev[1], p->stream);
    cudaEventRecord(p->ev[2], p->stream);
  }
  {
    const int64_t total = ncols * (int64_t)st->nrows;
    int64_t blocks = (total + 255) / 256;
    if (blocks > (int64_t)p->num_sms * 32) blocks = (int64_t)p->num_sms * 32;
    tc_reduce_kernel<<<(unsigned)blocks, 256, 0, p->stream>>>(st->partial, st->ksplit, p->n, st->nrows, st->l2p,
                                                               st->om_exp, st->a_exp_max, Y, ldy, ly, X, ldx, col0,
                                                               ncols);
    e = cudaGetLastError();
  }
  if (timing) cudaEventRecord(p->ev[1 + 2 * p->ev_panels], p->stream);
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


rid_status rid_tc_plan_init_fp64(rid_plan_s* p) { return rid_tc_plan_setup_fp64(p, 0); }

cudaError_t rid_tc_refresh_omega_fp64(const rid_plan_s* p) {
  const TcState* st = (const TcState*)p->tc_state;
  if (!st) return cudaErrorNotSupported;
  // the rows of the state (Omega, then the row probes), cut as at plan time;
  // the padding rows of the tiles keep the zeros of the setup
  return rid_tc_cut_omega(p->omega + (int64_t)st->row0 * p->ldo, p->ldo, p->m, st->nrows, st->KP, st->tile_w,
                          st->pair, st->om_exp, st->om_slices, p->num_sms, p->stream);
}
