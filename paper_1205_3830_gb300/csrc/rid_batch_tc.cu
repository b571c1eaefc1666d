// Batched sketches on the tensor cores: Y_p = Omega_p A_p and the row probes'
// X_p = G A_p (Sec. 2 and Sec. 3.3) for every problem p of a batch, FP64-grade
// by the exact-slice emulation of rid_sketch_tc.cu, in one persistent
// cooperative launch.
//
// The problems, largest first, are grouped into waves whose digit tiles fit
// one workspace buffer; two buffers alternate.  For each wave every CTA
//   1. cuts digits: every warp takes tasks of one column of A' x one
//      256-real chunk (the chunk's exponent, then its 7 balanced base-256
//      digits, stored in the swizzled tile image the product loads) or one
//      row of Omega' x one chunk, from one atomic counter per wave;
//   2. waits at a grid barrier: the wave's digits are complete;
//   3. multiplies its own list of (problem, N-tile, column block, K-split)
//      items, built on the host by longest-processing-time-first assignment,
//      through the warp-specialized tcgen05 pipeline of the plan's product
//      (bulk copies of pre-tiled digits, four TMEM accumulator groups, a
//      double-FP32 flush per chunk), and writes Y and X from the flush warps;
//      a problem split over K writes partial sums instead, and the CTA whose
//      split arrives last sums them in split order.
// Wave w + 1 is cut into the other buffer, so a CTA that finishes its products
// early goes straight on to the next wave's digits.
//
// The result of a problem does not depend on the waves, the CTAs or the other
// problems: every column chunk is summed in the same order as in the plan's
// product, and with one K-split a problem's Y has the bits a plan's sketch
// gives (the plan also runs one split for fewer than 16 chunks).
#include <algorithm>
#include <climits>
#include <queue>
#include <vector>

#include "rid_internal.cuh"
#include "rid_tc.cuh"
#include "rid_tc_digits.cuh"

using namespace rid_tc;

namespace {

constexpr int BTC_MAX_TILE_W = 128;
constexpr uint32_t BTC_A_STAGE = TC_S * TC_TILE_BYTES;                        // one stage's A tiles
constexpr uint32_t BTC_O_STAGE_MAX = TC_S * BTC_MAX_TILE_W * TC_KS * 2;       // the widest Omega tiles
constexpr uint32_t BTC_SLOT = BTC_A_STAGE + BTC_O_STAGE_MAX;
constexpr int BTC_SLOTS = 2;
constexpr int BTC_DYN_SMEM = BTC_SLOTS * BTC_SLOT + 1024;
static_assert(BTC_DYN_SMEM <= TC_DYN_SMEM_MAX, "two stages of the widest tiles must fit");
static_assert(TC_SPC * TC_S * 8 * 4 * 16 <= (int)BTC_SLOT, "the cutting atoms fit in one ring slot");
constexpr long long BTC_BARRIER_BUDGET = 8000000000ll;   // clock cycles (~4 s): a wave of the slowest CTA

struct BtcProb {
  const double2* A;
  int64_t lda, m, n;
  const double2* om;       // Omega': ls complex rows (l of Omega, then r probe rows), ld ldo
  int64_t ldo;
  const int* om_exp;       // [ls] row exponents
  double2* Y;
  int64_t ldy;
  double2* X;              // r x n, ld r
  int l, ls, r;
  int l2, ntiles, tile_w, l2p, NC, ksplit, cps, nblocks;
  int64_t nst;             // K stages
  int wave;
  int cnt_off;             // first K-split counter (ntiles x nblocks x flush warps of them) when ksplit > 1
  int64_t a_off, o_off, e_off, part_off;   // byte offsets in the wave's buffer
};

struct BtcItem {
  int32_t p;               // problem (position in the sorted order)
  int16_t nt, jb, ks, pad;
};

struct BtcArgs {
  const BtcProb* probs;
  const BtcItem* items;
  const int32_t* item_first;   // [waves * gridDim.x + 1]: items of (wave, CTA)
  const int32_t* wave_first;   // [waves + 1]: problems of each wave
  const int64_t* a_pref;       // [count + 1]: prefix of the A cutting tasks
  const int64_t* o_pref;       // [count + 1]: prefix of the Omega cutting tasks
  unsigned char* buf0;
  unsigned char* buf1;
  unsigned* ctr;               // [0] grid barrier, [1 + w] cutting tasks of wave w
  unsigned* split_cnt;
  int waves;
  int* err;
};

__device__ __forceinline__ unsigned char* wave_buf(const BtcArgs& a, int w) { return (w & 1) ? a.buf1 : a.buf0; }

// Largest p in [lo, hi) with pref[p] <= t.
__device__ __forceinline__ int find_prob(const int64_t* pref, int lo, int hi, int64_t t) {
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pref[mid] <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}

// 32 lanes x 8 consecutive 32-bit TMEM columns (as tmem_ld16, half as wide).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}

__device__ __forceinline__ void group_sync(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier on a monotonic counter (one thread per CTA): false when the
// wait ran out of its budget.
__device__ bool grid_arrive_wait(unsigned* ctr, unsigned target) {
  __threadfence();
  atomicAdd(ctr, 1u);
  if (ld_acquire(ctr) >= target) return true;
  const long long t0 = clock64();
  while (ld_acquire(ctr) < target) {
    if (clock64() - t0 > BTC_BARRIER_BUDGET) return false;
    __nanosleep(64);
  }
  return true;
}

// ---- cutting tasks -------------------------------------------------------------------
// One warp per task, no shared memory and no barriers: an A' task is one
// column x one 256-real chunk, an Omega' task one row x one chunk.  A lane
// takes 4 consecutive complex entries (reals 8 lane .. 8 lane + 7 of the
// chunk: one 16-byte piece of one K stage's tile row per digit) and stores its
// 7 pieces straight into the swizzled tile image; the 4 lanes of a stage
// write the row's 64 bytes, so every store fills whole sectors.  The wave's
// A' tasks come first in one task range, then its Omega' tasks; warps take
// them in grabs of BTC_GRAB from one atomic counter, requesting the next grab
// while working on the current one, and find a task's problem from the last
// task's range, so neither the atomic nor the search delays a task.  The next
// task's entries are loaded while the current one is cut.
constexpr int BTC_GRAB = 16;

struct TaskQueue {
  int64_t nxt, lim, pre;    // next task, end of the current grab, start of the requested one
  int p;                    // problem of the last task and its task range
  int64_t p_lo, p_hi;
};

// What cutting one wave reads, passed by value (kept in registers: a
// reference to the kernel's argument block would put it in local memory).
struct CutWave {
  const BtcProb* probs;
  const int64_t* a_pref;
  const int64_t* o_pref;
  unsigned char* buf;
  unsigned* ctr;
  int p_lo, p_hi;
  int64_t ta, tend;         // A' tasks, all tasks of the wave
};

__device__ __forceinline__ void queue_init(TaskQueue& q, unsigned* ctr) {
  q.nxt = (int64_t)atomicAdd(ctr, (unsigned)BTC_GRAB);
  q.lim = q.nxt + BTC_GRAB;
  q.pre = (int64_t)atomicAdd(ctr, (unsigned)BTC_GRAB);
  q.p = -1;
  q.p_lo = q.p_hi = 0;
}

// Next task's number within its problem (and kind) and the problem; p = -1
// past the wave's end.  Tasks below ta are A' tasks, the others Omega' tasks.
__device__ __forceinline__ int64_t queue_next(TaskQueue& q, const CutWave& cw, int& p) {
  if (q.nxt == q.lim) {
    q.nxt = q.pre;
    q.lim = q.pre + BTC_GRAB;
    q.pre = (int64_t)atomicAdd(cw.ctr, (unsigned)BTC_GRAB);
  }
  const int64_t t = q.nxt++;
  if (t >= cw.tend) {
    p = -1;
    return t;
  }
  if (t < q.p_lo || t >= q.p_hi) {
    // the problem's task range, in wave-relative task numbers
    if (t < cw.ta) {
      const int64_t base = cw.a_pref[cw.p_lo];
      q.p = find_prob(cw.a_pref, cw.p_lo, cw.p_hi, base + t);
      q.p_lo = cw.a_pref[q.p] - base;
      q.p_hi = cw.a_pref[q.p + 1] - base;
    } else {
      const int64_t base = cw.o_pref[cw.p_lo];
      q.p = find_prob(cw.o_pref, cw.p_lo, cw.p_hi, base + (t - cw.ta));
      q.p_lo = cw.ta + cw.o_pref[q.p] - base;
      q.p_hi = cw.ta + cw.o_pref[q.p + 1] - base;
    }
  }
  p = q.p;
  return t - q.p_lo;
}

struct CutTask {
  int p;                    // problem; -1: none
  bool omega;               // an Omega' task (else A')
  int c;                    // chunk
  int idx;                  // column j of A' / row i of Omega
};

// A' task number = c n + j (chunk-major); Omega' task number = i NC + c.
// Decoded once by lane 0 (32-bit division: a problem has fewer than 2^31
// tasks) and broadcast.
__device__ __forceinline__ void cut_decode(const CutWave& cw, int p, bool omega, int64_t local, CutTask& t) {
  t.p = p;
  t.omega = omega;
  t.c = t.idx = 0;
  if (p < 0) return;
  const BtcProb& P = cw.probs[p];
  const unsigned u = (unsigned)local;
  if (!omega) {
    const unsigned n = (unsigned)P.n;
    t.c = (int)(u / n);
    t.idx = (int)(u - (unsigned)t.c * n);
  } else {
    const unsigned nc = (unsigned)P.NC;
    t.idx = (int)(u / nc);
    t.c = (int)(u - (unsigned)t.idx * nc);
  }
}

__device__ __forceinline__ void cut_load(const CutWave& cw, const CutTask& t, int lane, double2 (&x)[4]) {
  if (t.p < 0) return;
  const BtcProb& P = cw.probs[t.p];
  const double2* src = !t.omega ? P.A + (int64_t)t.idx * P.lda : P.om + (int64_t)t.idx * P.ldo;
  const int64_t r0 = (int64_t)t.c * 128 + 4 * lane;
#pragma unroll
  for (int u = 0; u < 4; ++u) x[u] = r0 + u < P.m ? __ldg(src + r0 + u) : make_double2(0.0, 0.0);
}

__device__ __forceinline__ void store_pieces(uint16_t* base, int64_t tile_elems, int off, const uint32_t (&w)[4][TC_S]) {
#pragma unroll
  for (int s = 0; s < TC_S; ++s)
    *(uint4*)(base + s * tile_elems + off) = make_uint4(w[0][s], w[1][s], w[2][s], w[3][s]);
}

// -x by its sign bit (no FP64 instruction)
__device__ __forceinline__ double neg_bits(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

__device__ __forceinline__ void cut_store(const CutWave& cw, const CutTask& t, int lane, const double2 (&x)[4]) {
  const BtcProb& P = cw.probs[t.p];
  const int st_in_chunk = lane >> 2;
  const int k = 8 * (lane & 3);
  const int c = t.c;
  uint32_t wd[4][TC_S];
  if (!t.omega) {
    const int64_t j = t.idx;
    int e = TC_EXP_ZERO;
#pragma unroll
    for (int u = 0; u < 4; ++u) e = max(e, max(exp_of(x[u].x), exp_of(x[u].y)));
    e = __reduce_max_sync(0xffffffffu, e);
#pragma unroll
    for (int u = 0; u < 4; ++u) digit_words(x[u], e, wd[u]);
    // tiles [column block][K stage][digit] of 128 rows; column j is row j % 128
    uint16_t* base = (uint16_t*)(cw.buf + P.a_off) +
                     (((j >> 7) * P.nst + (int64_t)c * TC_SPC + st_in_chunk) * TC_S) * TC_TILE_ELEMS;
    store_pieces(base, TC_TILE_ELEMS, tile_offset((int)(j & 127), k) / 2, wd);
    if (lane == 0) ((int*)(cw.buf + P.e_off))[j * P.NC + c] = e;
  } else {
    const int i = t.idx;
    const int e = P.om_exp[i];
    // Omega' row 2i: (Re w, -Im w); row 2i + 1: (Im w, Re w)
    const int R = 2 * i, nt = R / P.tile_w, rr = R - nt * P.tile_w;
    const int64_t tile_elems = (int64_t)P.tile_w * TC_KS;
    uint16_t* base = (uint16_t*)(cw.buf + P.o_off) +
                     (((int64_t)nt * P.nst + (int64_t)c * TC_SPC + st_in_chunk) * TC_S) * tile_elems;
#pragma unroll
    for (int u = 0; u < 4; ++u) digit_words(make_double2(x[u].x, neg_bits(x[u].y)), e, wd[u]);
    store_pieces(base, tile_elems, tile_offset(rr, k) / 2, wd);
#pragma unroll
    for (int u = 0; u < 4; ++u) digit_words(make_double2(x[u].y, x[u].x), e, wd[u]);
    store_pieces(base, tile_elems, tile_offset(rr + 1, k) / 2, wd);
  }
}

// All 16 warps cut one wave's digits.
// (out of line: its registers are allocated apart from the product's flush loop)
__device__ __noinline__ void cut_wave(const CutWave cw) {
  const int lane = threadIdx.x & 31;
  TaskQueue q;
  CutTask cur{-1, false, 0, 0}, nxt{-1, false, 0, 0};
  auto next = [&](CutTask& dst) {
    CutTask t{-1, false, 0, 0};
    if (lane == 0) {
      int p = -1;
      const int64_t local = queue_next(q, cw, p);
      cut_decode(cw, p, q.p_lo >= cw.ta, local, t);
    }
    dst.p = __shfl_sync(0xffffffffu, t.p, 0);
    dst.omega = __shfl_sync(0xffffffffu, (int)t.omega, 0) != 0;
    dst.c = __shfl_sync(0xffffffffu, t.c, 0);
    dst.idx = __shfl_sync(0xffffffffu, t.idx, 0);
  };
  if (lane == 0) queue_init(q, cw.ctr);
  next(cur);
  double2 x[4], xn[4];
  cut_load(cw, cur, lane, x);
  while (cur.p >= 0) {
    next(nxt);
    cut_load(cw, nxt, lane, xn);
    cut_store(cw, cur, lane, x);
    cur = nxt;
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = xn[u];
  }
}

// Y or X entry (i, j) of a problem from the (hi, lo) sums of Omega' rows 2i and
// 2i + 1 (re, im), as the plan's reduction forms it.
__device__ __forceinline__ void store_entry(const BtcProb& P, int64_t j, int ii, int ea, double re, double im) {
  const int ex = P.om_exp[ii];
  const double2 v = make_double2(ea == TC_EXP_ZERO ? 0.0 : ldexp(re, ex + ea - 16),
                                 ea == TC_EXP_ZERO ? 0.0 : ldexp(im, ex + ea - 16));
  if (ii < P.l) P.Y[ii + j * P.ldy] = v;
  else P.X[(ii - P.l) + j * P.r] = v;
}

__global__ void __launch_bounds__(TC_THREADS, 1) batch_sketch_tc_kernel(BtcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* ring = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full_bar[BTC_SLOTS], empty_bar[BTC_SLOTS];
  __shared__ uint64_t acc_full[TC_G], acc_empty[TC_G], mma_done;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 13) tmem_alloc(&tmem_slot, 512);
  if (threadIdx.x == 0) {
    for (int i = 0; i < BTC_SLOTS; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&empty_bar[i], 1);
    }
    for (int g = 0; g < TC_G; ++g) {
      mbar_init(&acc_full[g], 1);
      mbar_init(&acc_empty[g], TC_FLUSH_WARPS);
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
  // stage / chunk counters of each role, continued across items and waves
  uint32_t pit = 0, mit = 0, mcl = 0, fcl = 0;
  for (int w = 0; w < a.waves; ++w) {
    // ---------------- 1. cut wave w's digits ----------------
    {
      const int p_lo = a.wave_first[w], p_hi = a.wave_first[w + 1];
      const int64_t ta = a.a_pref[p_hi] - a.a_pref[p_lo];
      cut_wave(CutWave{a.probs, a.a_pref, a.o_pref, wave_buf(a, w), a.ctr + 1 + w, p_lo, p_hi, ta,
                       ta + a.o_pref[p_hi] - a.o_pref[p_lo]});
    }
    fence_proxy_async_global();          // the digits are read by other CTAs' bulk copies
    __syncthreads();
    // ---------------- 2. every CTA's digits of the wave are in place ----------------
    if (threadIdx.x == 0 && !grid_arrive_wait(a.ctr, (unsigned)(w + 1) * gridDim.x)) fail(41);
    __syncthreads();
    if (s_abort) break;
    fence_proxy_async_smem();            // the ring's generic use (cutting atoms) ends here
    __syncthreads();
    // ---------------- 3. this CTA's items of the wave ----------------
    const int q0 = a.item_first[w * gridDim.x + blockIdx.x], q1 = a.item_first[w * gridDim.x + blockIdx.x + 1];
    unsigned char* buf = wave_buf(a, w);
    if (warp == 12) {
      if (lane == 0) {
        // ---- producer: the stages' A and Omega tiles, one bulk copy each ----
        fence_proxy_async_global();
        const uint32_t pit0 = pit;
        for (int q = q0; q < q1 && !s_abort; ++q) {
          const BtcItem it = a.items[q];
          const BtcProb& P = a.probs[it.p];
          const int c_begin = it.ks * P.cps, c_end = min(P.NC, c_begin + P.cps);
          const int stages = (c_end - c_begin) * TC_SPC;
          const uint32_t o_bytes = (uint32_t)(TC_S * P.tile_w * TC_KS * 2);
          const unsigned char* a_src = buf + P.a_off + ((int64_t)it.jb * P.nst + (int64_t)c_begin * TC_SPC) * BTC_A_STAGE;
          const unsigned char* o_src = buf + P.o_off + ((int64_t)it.nt * P.nst + (int64_t)c_begin * TC_SPC) * o_bytes;
          for (int s = 0; s < stages; ++s) {
            const uint32_t slot = pit & 1u, round = pit >> 1;
            if (round > 0 && !mbar_wait(&empty_bar[slot], (round - 1) & 1u, TC_WAIT_BUDGET)) {
              fail(11);
              break;
            }
            mbar_arrive_expect_tx(&full_bar[slot], BTC_A_STAGE + o_bytes);
            bulk_load(ring + slot * BTC_SLOT, a_src, BTC_A_STAGE, &full_bar[slot]);
            bulk_load(ring + slot * BTC_SLOT + BTC_A_STAGE, o_src, o_bytes, &full_bar[slot]);
            a_src += BTC_A_STAGE;
            o_src += o_bytes;
            ++pit;
          }
        }
        // the ring is free again once the MMAs released every stage (or, after
        // an error, once every copy issued into it has landed)
        for (uint32_t k = pit - pit0 > 2 ? pit - 2 : pit0; k < pit; ++k) {
          const bool ok = s_abort ? mbar_wait(&full_bar[k & 1u], (k >> 1) & 1u, TC_WAIT_BUDGET)
                                  : mbar_wait(&empty_bar[k & 1u], (k >> 1) & 1u, TC_WAIT_BUDGET);
          if (!ok) fail(12);
        }
      }
    } else if (warp == 13) {
      // ---- MMA issuer: the whole warp runs the loop, one elected lane issues ----
      for (int q = q0; q < q1 && !s_abort; ++q) {
        const BtcItem it = a.items[q];
        const BtcProb& P = a.probs[it.p];
        const int c_begin = it.ks * P.cps, c_end = min(P.NC, c_begin + P.cps);
        const uint32_t idesc = idesc_bf16_f32(128, tile_mma_n(P.tile_w, P.l2, it.nt, false));
        const uint64_t o_step = (uint64_t)(P.tile_w * TC_KS * 2) >> 4;
        for (int c = c_begin; c < c_end && !s_abort; ++c, ++mcl) {
          for (int b = 0; b < TC_SPC; ++b) {
            const uint32_t slot = mit & 1u, round = mit >> 1;
            if (!__all_sync(0xffffffffu, mbar_wait(&full_bar[slot], round & 1u, TC_WAIT_BUDGET))) {
              if (lane == 0) fail(21);
              break;
            }
            tc_fence_after();
            const uint64_t da0 = tile_desc(ring + slot * BTC_SLOT), db0 = tile_desc(ring + slot * BTC_SLOT + BTC_A_STAGE);
            if (!mma_stage<TC_S, false>(tmem, da0, db0, o_step, idesc, b, (int)mcl, TC_SPC, acc_empty, acc_full)) {
              if (lane == 0) fail(22);
              break;
            }
            mma_commit_w(&empty_bar[slot]);
            ++mit;
          }
        }
      }
    } else if (warp < TC_FLUSH_WARPS) {
      // ---- flush warps: TMEM lanes 32 (w % 4) .. + 31, tile columns 48 (w / 4) .. ----
      const int quarter = warp & 3, third = warp >> 2;
      const int col0 = third * 48;
      const int nblk = third < 2 ? 3 : 2;
      const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col0;
      for (int q = q0; q < q1 && !s_abort; ++q) {
        const BtcItem it = a.items[q];
        const BtcProb& P = a.probs[it.p];
        const int c_begin = it.ks * P.cps, c_end = min(P.NC, c_begin + P.cps);
        const int64_t j = (int64_t)it.jb * 128 + quarter * 32 + lane;
        const bool j_ok = j < P.n;
        // exponents written by other CTAs in this launch: read through L2
        const int* a_exp = (const int*)(buf + P.e_off) + j * P.NC;
        int emax = TC_EXP_ZERO;
        if (j_ok)
          for (int c = 0; c < P.NC; ++c) emax = max(emax, __ldcg(a_exp + c));
        const int row0 = it.nt * P.tile_w;
        const int n_tile = min(P.tile_w, P.l2 - row0);
        const int nb = max(0, min(nblk, (n_tile - col0 + 15) / 16));   // 16-column blocks holding rows
        float hi[48], lo[48];
#pragma unroll
        for (int i = 0; i < 48; ++i) {
          hi[i] = 0.f;
          lo[i] = 0.f;
        }
        for (int c = c_begin; c < c_end && !s_abort; ++c, ++fcl) {
          const int e = j_ok ? __ldcg(a_exp + c) : TC_EXP_ZERO;
          const int delta = e - emax;
          const float scale = delta >= -126 ? __int_as_float((127 + delta) << 23) : 0.f;
          for (int gi = 0; gi < TC_G; ++gi) {
            const int g = TC_G - 1 - gi;
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[g], fcl & 1u, TC_WAIT_BUDGET));
            if (!ok) {
              if (lane == 0) fail(31);
              break;
            }
            tc_fence_after();
            if (nb == 0) {                 // no rows of this warp in the tile: release at once
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(&acc_empty[g]);
            }
#pragma unroll
            for (int h8 = 0; h8 < 6; ++h8) {          // 8 columns at a time: fewer registers in flight
              if (h8 < 2 * nb) {
                uint32_t r[8];
                tmem_ld8(lane_base + (uint32_t)(g * 128 + h8 * 8), r);
                tmem_ld_wait();
                if (h8 == 2 * nb - 1) {        // all columns read: the group may be overwritten
                  tc_fence_before();
                  __syncwarp();
                  if (lane == 0) mbar_arrive(&acc_empty[g]);
                }
#pragma unroll
                for (int qq = 0; qq < 8; ++qq) {
                  const int i = h8 * 8 + qq;
                  const float v = __fmul_rn(__uint_as_float(r[qq]), scale);
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
        if (s_abort) break;
        if (P.ksplit == 1) {
          if (j_ok) {
#pragma unroll
            for (int i = 0; i < 48; i += 2) {
              if (i < nb * 16 && col0 + i < n_tile) {
                const double re = 0.0 + ((double)hi[i] + (double)lo[i]);
                const double im = 0.0 + ((double)hi[i + 1] + (double)lo[i + 1]);
                store_entry(P, j, (row0 + col0 + i) >> 1, emax, re, im);
              }
            }
          }
        } else {
          // partial sums of this split; per warp, the split that arrives last
          // sums all of them in split order
          float2* part = (float2*)(buf + P.part_off);
          if (j_ok) {
            float2* dst = part + ((int64_t)it.ks * P.n + j) * P.l2p + row0 + col0;
#pragma unroll
            for (int i = 0; i < 48; ++i)
              if (i < nb * 16 && col0 + i < n_tile) dst[i] = make_float2(hi[i], lo[i]);
          }
          __threadfence();
          __syncwarp();
          unsigned last = 0;
          if (lane == 0)
            last = atomicAdd(a.split_cnt + P.cnt_off + (it.nt * P.nblocks + it.jb) * TC_FLUSH_WARPS + warp, 1u) ==
                   (unsigned)(P.ksplit - 1);
          last = __shfl_sync(0xffffffffu, last, 0);
          if (last) {
            __threadfence();
            if (j_ok) {
              const int64_t split_stride = P.n * (int64_t)P.l2p;
              const float2* src = part + j * P.l2p + row0 + col0;
#pragma unroll 1
              for (int i = 0; i < 48; i += 2) {
                if (i < nb * 16 && col0 + i < n_tile) {
                  double re = 0.0, im = 0.0;
                  for (int s = 0; s < P.ksplit; ++s) {
                    const float4 v = __ldcg((const float4*)(src + s * split_stride + i));
                    re += (double)v.x + (double)v.y;
                    im += (double)v.z + (double)v.w;
                  }
                  store_entry(P, j, (row0 + col0 + i) >> 1, emax, re, im);
                }
              }
            }
          }
        }
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (s_abort) break;
  }

  // ---------------- teardown ----------------
  __syncthreads();
  if (warp == 13) {
    mma_commit_w(&mma_done);
    __syncwarp();
    if (!mbar_wait(&mma_done, 0, TC_WAIT_BUDGET)) fail(91);
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ---- batch setup kernels ------------------------------------------------------------------
// Omega' of every problem: rows 0 .. l-1 from the problem's seed (the plan's
// Omega), rows l .. ls-1 from the probe seed (the plan's row probes); the
// Philox counters of a plan.  Blocks (problem, slice of the entries).
__global__ void batch_omega_kernel(const BtcProb* __restrict__ probs, uint64_t* __restrict__ seeds,
                                   uint64_t probe_seed) {
  const BtcProb P = probs[blockIdx.x];
  const uint64_t seed = seeds[blockIdx.x];
  const int64_t total = (int64_t)P.ls * P.m;
  double2* om = const_cast<double2*>(P.om);
  for (int64_t e = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.y * blockDim.x) {
    const int64_t i = e / P.m, j = e - i * P.m;
    om[i * P.ldo + j] = i < P.l ? philox_complex_normal((uint64_t)i, (uint64_t)j, seed, RID_STREAM_OMEGA)
                                : philox_complex_normal((uint64_t)(i - P.l), (uint64_t)j, probe_seed,
                                                        RID_STREAM_LPROBES);
  }
}

// Row exponents of Omega' (as the plan's Omega exponent pass) and the probe
// rows' squared norms ||g_q||^2 (fixed-order sums).  Block (p, i): row i of
// problem p.
__global__ void __launch_bounds__(256) batch_omega_rows_kernel(const BtcProb* __restrict__ probs,
                                                               double* const* __restrict__ g_norm2) {
  __shared__ int red[8];
  __shared__ double dred[8];
  const BtcProb P = probs[blockIdx.x];
  const int i = blockIdx.y;
  if (i >= P.ls) return;
  const double2* row = P.om + (int64_t)i * P.ldo;
  int e = TC_EXP_ZERO;
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < P.m; r += blockDim.x) {
    const double2 w = row[r];
    e = max(e, max(exp_of(w.x), exp_of(w.y)));
    s += w.x * w.x + w.y * w.y;
  }
  e = __reduce_max_sync(0xffffffffu, e);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = e;
    dred[threadIdx.x >> 5] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int v = red[0];
    double t = dred[0];
    for (int w = 1; w < 8; ++w) {
      v = max(v, red[w]);
      t += dred[w];
    }
    const_cast<int*>(P.om_exp)[i] = v;
    if (i >= P.l) g_norm2[blockIdx.x][i - P.l] = t;
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------
struct rid_btc_s {
  int device;
  int count;                  // problems
  int nprobe;
  int grid;                   // CTAs of the persistent launch (one per SM)
  int waves;
  int64_t nitems;
  char* dev;                  // descriptors, work lists, counters, Omega', exponents, X, norms
  unsigned char* bufs;        // the two wave buffers
  size_t dev_bytes, buf_bytes;
  size_t clear_off, clear_bytes;   // counters and error word, cleared before every run
  BtcArgs args;
  std::vector<double2*> X;    // per problem (input order)
  std::vector<double*> gn2;
  int* err;
};

namespace {

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
size_t al1k(size_t x) { return (x + 1023) & ~(size_t)1023; }

}  // namespace

rid_status rid_btc_create(rid_btc_s** out, const rid_btc_problem* in, int32_t count, int32_t nprobe,
                          uint64_t probe_seed, size_t wave_bytes, cudaStream_t stream) {
  *out = nullptr;
  if (count < 1 || nprobe < 1 || nprobe > RID_MAX_PROBES) return RID_EINVAL;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return RID_ECUDA;
  int sms = 0, coop = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
  if (sms < 1 || !coop) return RID_EUNSUPPORTED;
  {
    // one CTA (512 threads, two ring stages) must fit on an SM
    if (cudaFuncSetAttribute(batch_sketch_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_DYN_SMEM_MAX) !=
        cudaSuccess)
      return RID_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_sketch_tc_kernel, TC_THREADS, BTC_DYN_SMEM) !=
            cudaSuccess ||
        per_sm < 1)
      return RID_EUNSUPPORTED;
  }
  const int G = sms;

  // ---- per-problem shapes, tiles and byte counts ----
  std::vector<BtcProb> P((size_t)count);
  std::vector<int64_t> bytes((size_t)count), a_tasks((size_t)count), o_tasks((size_t)count);
  for (int32_t i = 0; i < count; ++i) {
    const rid_btc_problem& x = in[i];
    BtcProb& b = P[i];
    b = BtcProb{};
    b.A = x.A;
    b.lda = x.lda;
    b.m = x.m;
    b.n = x.n;
    b.Y = x.Y;
    b.ldy = x.ldy;
    b.l = x.l;
    b.r = nprobe;
    b.ls = x.l + nprobe;
    b.l2 = 2 * b.ls;
    const int nmax = x.tile_n >= 16 && x.tile_n <= BTC_MAX_TILE_W ? x.tile_n / 16 * 16 : BTC_MAX_TILE_W;
    b.ntiles = (int)cdiv(b.l2, nmax);
    b.tile_w = (int)cdiv(cdiv(b.l2, b.ntiles), 16) * 16;
    if (b.tile_w > BTC_MAX_TILE_W) return RID_EUNSUPPORTED;
    b.l2p = b.ntiles * b.tile_w;
    b.NC = (int)cdiv(2 * b.m, TC_KC);
    b.nst = (int64_t)b.NC * TC_SPC;
    b.nblocks = (int)cdiv(b.n, 128);
    const int ks = x.ksplit >= 1 ? std::min(x.ksplit, b.NC) : 1;
    b.cps = (int)cdiv(b.NC, ks);
    b.ksplit = (int)cdiv(b.NC, b.cps);
    if (b.ntiles > 32767 || b.nblocks > 32767 || b.ksplit > 32767) return RID_EUNSUPPORTED;
    const int64_t a_b = (int64_t)b.nblocks * b.nst * BTC_A_STAGE;
    const int64_t o_b = (int64_t)b.ntiles * b.nst * TC_S * b.tile_w * TC_KS * 2;
    const int64_t e_b = b.n * (int64_t)b.NC * 4;
    const int64_t p_b = b.ksplit > 1 ? (int64_t)b.ksplit * b.n * b.l2p * 8 : 0;
    b.a_off = 0;
    b.o_off = (int64_t)al1k(a_b);
    b.e_off = b.o_off + (int64_t)al1k(o_b);
    b.part_off = b.e_off + (int64_t)al1k(e_b);
    bytes[i] = b.part_off + (int64_t)al1k(p_b);
    a_tasks[i] = (int64_t)b.NC * b.n;
    o_tasks[i] = (int64_t)b.ls * b.NC;
  }
  // ---- order (largest first) and waves ----
  std::vector<int32_t> order((size_t)count);
  for (int32_t i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return bytes[x] > bytes[y]; });
  int64_t W = (int64_t)wave_bytes;
  if (W <= 0) W = (int64_t)2 << 30;
  W = std::max<int64_t>(W, bytes[order[0]]);
  std::vector<int32_t> wave_first{0};
  int64_t cur = 0, buf_need = 0;
  for (int32_t t = 0; t < count; ++t) {
    const int32_t i = order[t];
    if (cur > 0 && cur + bytes[i] > W) {
      wave_first.push_back(t);
      cur = 0;
    }
    // offsets within the wave's buffer
    P[i].a_off += cur;
    P[i].o_off += cur;
    P[i].e_off += cur;
    P[i].part_off += cur;
    P[i].wave = (int)wave_first.size() - 1;
    cur += bytes[i];
    buf_need = std::max(buf_need, cur);
  }
  wave_first.push_back(count);
  const int waves = (int)wave_first.size() - 1;

  // ---- work lists: per wave, items assigned longest first to the least-loaded CTA ----
  std::vector<BtcItem> items;
  std::vector<int32_t> item_first;
  item_first.reserve((size_t)waves * G + 1);
  int split_counters = 0;
  std::vector<BtcProb> sorted((size_t)count);
  for (int32_t t = 0; t < count; ++t) {
    sorted[t] = P[order[t]];
    if (sorted[t].ksplit > 1) {
      sorted[t].cnt_off = split_counters;
      split_counters += sorted[t].ntiles * sorted[t].nblocks * TC_FLUSH_WARPS;
    }
  }
  for (int w = 0; w < waves; ++w) {
    struct Cand {
      double cost;
      BtcItem it;
    };
    std::vector<Cand> cands;
    for (int32_t t = wave_first[w]; t < wave_first[w + 1]; ++t) {
      const BtcProb& b = sorted[t];
      for (int nt = 0; nt < b.ntiles; ++nt)
        for (int jb = 0; jb < b.nblocks; ++jb)
          for (int ks = 0; ks < b.ksplit; ++ks) {
            const int c_begin = ks * b.cps, c_end = std::min(b.NC, c_begin + b.cps);
            // bytes moved per stage (the bound), plus a fixed cost per item
            const double cost = (double)(c_end - c_begin) * TC_SPC * (BTC_A_STAGE + TC_S * b.tile_w * TC_KS * 2) +
                                2.0 * BTC_SLOT;
            cands.push_back({cost, BtcItem{t, (int16_t)nt, (int16_t)jb, (int16_t)ks, 0}});
          }
    }
    std::stable_sort(cands.begin(), cands.end(), [](const Cand& x, const Cand& y) { return x.cost > y.cost; });
    std::vector<std::vector<BtcItem>> lists((size_t)G);
    using Load = std::pair<double, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int b = 0; b < G; ++b) heap.push({0.0, b});
    for (const Cand& c : cands) {
      Load l = heap.top();
      heap.pop();
      lists[l.second].push_back(c.it);
      l.first += c.cost;
      heap.push(l);
    }
    for (int b = 0; b < G; ++b) {
      item_first.push_back((int32_t)items.size());
      items.insert(items.end(), lists[b].begin(), lists[b].end());
    }
  }
  item_first.push_back((int32_t)items.size());
  std::vector<int64_t> a_pref((size_t)count + 1, 0), o_pref((size_t)count + 1, 0);
  for (int32_t t = 0; t < count; ++t) {
    a_pref[t + 1] = a_pref[t] + a_tasks[order[t]];
    o_pref[t + 1] = o_pref[t] + o_tasks[order[t]];
  }

  // ---- device memory ----
  size_t total = 0;
  auto take = [&](size_t b) { const size_t at = total; total += al1k(b); return at; };
  const size_t off_probs = take(sizeof(BtcProb) * (size_t)count);
  const size_t off_items = take(sizeof(BtcItem) * std::max<size_t>(items.size(), 1));
  const size_t off_ifirst = take(sizeof(int32_t) * item_first.size());
  const size_t off_wfirst = take(sizeof(int32_t) * wave_first.size());
  const size_t off_apref = take(sizeof(int64_t) * a_pref.size());
  const size_t off_opref = take(sizeof(int64_t) * o_pref.size());
  const size_t off_seeds = take(sizeof(uint64_t) * (size_t)count);
  const size_t off_gptr = take(sizeof(double*) * (size_t)count);
  const size_t clear_bytes = sizeof(unsigned) * (1 + (size_t)waves + (size_t)split_counters) + sizeof(int);
  const size_t off_clear = take(clear_bytes);
  std::vector<size_t> off_om((size_t)count), off_exp((size_t)count), off_x((size_t)count), off_g((size_t)count);
  for (int32_t t = 0; t < count; ++t) {
    const BtcProb& b = sorted[t];
    off_om[t] = take(sizeof(double2) * (size_t)b.ls * (size_t)b.m);
    off_exp[t] = take(sizeof(int) * (size_t)b.ls);
    off_x[t] = take(sizeof(double2) * (size_t)nprobe * (size_t)b.n);
    off_g[t] = take(sizeof(double) * (size_t)nprobe);
  }
  rid_btc_s* h = new (std::nothrow) rid_btc_s();
  if (!h) return RID_ENOMEM;
  h->device = device;
  h->count = count;
  h->nprobe = nprobe;
  h->grid = G;
  h->waves = waves;
  h->nitems = (int64_t)items.size();
  h->dev_bytes = total;
  h->buf_bytes = al1k((size_t)buf_need);
  h->X.assign((size_t)count, nullptr);
  h->gn2.assign((size_t)count, nullptr);
  if (rid_dev_alloc((void**)&h->dev, total, stream, device) != cudaSuccess) {
    delete h;
    return RID_ENOMEM;
  }
  if (rid_dev_alloc((void**)&h->bufs, 2 * h->buf_bytes, stream, device) != cudaSuccess) {
    rid_dev_free(h->dev, stream);
    delete h;
    return RID_ENOMEM;
  }
  char* d = h->dev;
  std::vector<uint64_t> seeds((size_t)count);
  std::vector<double*> gptr((size_t)count);
  for (int32_t t = 0; t < count; ++t) {
    BtcProb& b = sorted[t];
    const int32_t i = order[t];
    b.om = (const double2*)(d + off_om[t]);
    b.ldo = b.m;
    b.om_exp = (const int*)(d + off_exp[t]);
    b.X = (double2*)(d + off_x[t]);
    seeds[t] = in[i].seed;
    gptr[t] = (double*)(d + off_g[t]);
    h->X[i] = b.X;
    h->gn2[i] = gptr[t];
  }
  h->clear_off = off_clear;
  h->clear_bytes = clear_bytes;
  h->err = (int*)(d + off_clear + clear_bytes - sizeof(int));
  BtcArgs& A = h->args;
  A.probs = (const BtcProb*)(d + off_probs);
  A.items = (const BtcItem*)(d + off_items);
  A.item_first = (const int32_t*)(d + off_ifirst);
  A.wave_first = (const int32_t*)(d + off_wfirst);
  A.a_pref = (const int64_t*)(d + off_apref);
  A.o_pref = (const int64_t*)(d + off_opref);
  A.buf0 = h->bufs;
  A.buf1 = h->bufs + h->buf_bytes;
  A.ctr = (unsigned*)(d + off_clear);
  A.split_cnt = A.ctr + 1 + waves;
  A.waves = waves;
  A.err = h->err;

  cudaError_t e = cudaMemcpyAsync(d + off_probs, sorted.data(), sizeof(BtcProb) * (size_t)count,
                                  cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpyAsync(d + off_items, items.data(), sizeof(BtcItem) * items.size(), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d + off_ifirst, item_first.data(), sizeof(int32_t) * item_first.size(), cudaMemcpyHostToDevice,
                        stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d + off_wfirst, wave_first.data(), sizeof(int32_t) * wave_first.size(), cudaMemcpyHostToDevice,
                        stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d + off_apref, a_pref.data(), sizeof(int64_t) * a_pref.size(), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d + off_opref, o_pref.data(), sizeof(int64_t) * o_pref.size(), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d + off_seeds, seeds.data(), sizeof(uint64_t) * seeds.size(), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d + off_gptr, gptr.data(), sizeof(double*) * gptr.size(), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d + off_clear, 0, clear_bytes, stream);
  // zero digits everywhere once: tile rows and columns that no task writes
  // (padding) are multiplied but never read back
  if (e == cudaSuccess) e = cudaMemsetAsync(h->bufs, 0, 2 * h->buf_bytes, stream);
  if (e == cudaSuccess) {
    int64_t most = 0;
    int max_ls = 0;
    for (const BtcProb& b : sorted) {
      most = std::max<int64_t>(most, (int64_t)b.ls * b.m);
      max_ls = std::max(max_ls, b.ls);
    }
    const unsigned gx = (unsigned)std::min<int64_t>(cdiv(most, 256), 64);
    batch_omega_kernel<<<dim3((unsigned)count, gx), 256, 0, stream>>>(A.probs, (uint64_t*)(d + off_seeds),
                                                                      probe_seed);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
      batch_omega_rows_kernel<<<dim3((unsigned)count, (unsigned)max_ls), 256, 0, stream>>>(A.probs,
                                                                                          (double* const*)(d + off_gptr));
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);     // the host arrays are pageable
  if (e != cudaSuccess) {
    rid_btc_destroy(h, stream);
    return RID_ECUDA;
  }
  *out = h;
  return RID_OK;
}

cudaError_t rid_btc_launch(const rid_btc_s* h, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(h->dev + h->clear_off, 0, h->clear_bytes, stream);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3((unsigned)h->grid);
  cfg.blockDim = dim3(TC_THREADS);
  cfg.dynamicSmemBytes = BTC_DYN_SMEM;
  cfg.stream = stream;
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, batch_sketch_tc_kernel, h->args);
}

const double2* rid_btc_x(const rid_btc_s* h, int32_t i) { return h->X[(size_t)i]; }
const double* rid_btc_gnorm2(const rid_btc_s* h, int32_t i) { return h->gn2[(size_t)i]; }
const int* rid_btc_error_word(const rid_btc_s* h) { return h->err; }

void rid_btc_info(const rid_btc_s* h, double out[4]) {
  out[0] = (double)(h->dev_bytes + 2 * h->buf_bytes);
  out[1] = (double)h->waves;
  out[2] = (double)h->nitems;
  out[3] = (double)h->grid;
}

void rid_btc_destroy(rid_btc_s* h, cudaStream_t stream) {
  if (!h) return;
  if (h->bufs) rid_dev_free(h->bufs, stream);
  if (h->dev) rid_dev_free(h->dev, stream);
  delete h;
}
