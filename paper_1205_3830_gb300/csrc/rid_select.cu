// Truncated QR with column pivoting of the sketch Y (Sec. 2, "Y ~= Q R", with
// the column permutation chosen by Businger-Golub pivoting).
//
// Two launch schemes share one column update (reflect_column / reflect_pair):
// a warp applies H_j^H to trailing columns, keeping each column in registers
// between the dot product and the update, and recomputes its remaining norm
// sum_{i>j} |Y_ic|^2 exactly.  Ties of the pivot norms go to the lowest column
// index; reflectors follow LAPACK's zlarfg convention.
//   - Plans by default: all k steps in one cooperative launch with a bounded
//     grid barrier per step (select_coop_kernel, below).
//   - The allocation-free entry, plans set to it (rid_plan_set_select_grid
//     with 0) and devices without cooperative launch: one launch per step;
//     the last CTA to finish (a fence and an atomic ticket, so no CTA waits on
//     another) reduces the posted (norm, column) pairs, swaps the pivot column
//     into place and forms the next reflector.
#include <climits>

#include "rid_internal.cuh"
#include "rid_tc.cuh"

namespace {

constexpr int QR_THREADS = 256;
constexpr int QR_WARPS = QR_THREADS / 32;
constexpr int QR_PER_LANE = 16;            // rows per lane kept in registers: l <= 512

struct ArgMax {
  double v;
  int i;
};

__device__ __forceinline__ ArgMax better(ArgMax a, ArgMax b) {
  return (b.v > a.v || (b.v == a.v && b.i < a.i)) ? b : a;
}

__device__ __forceinline__ ArgMax warp_argmax(ArgMax a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    ArgMax o;
    o.v = __shfl_xor_sync(0xffffffffu, a.v, off);
    o.i = __shfl_xor_sync(0xffffffffu, a.i, off);
    a = better(a, o);
  }
  return a;
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  return x;
}

// Block-wide argmax; result valid in every thread.
__device__ ArgMax block_argmax(ArgMax a) {
  __shared__ ArgMax red[QR_WARPS];
  __shared__ ArgMax result;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  a = warp_argmax(a);
  if (lane == 0) red[warp] = a;
  __syncthreads();
  if (warp == 0) {
    ArgMax b = lane < QR_WARPS ? red[lane] : ArgMax{-1.0, INT_MAX};
    b = warp_argmax(b);
    if (lane == 0) result = b;
  }
  __syncthreads();
  return result;
}

// Block-wide sum in a fixed order; result valid in every thread.
__device__ double block_sum(double x) {
  __shared__ double red[QR_WARPS];
  __shared__ double result;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  x = warp_sum(x);
  if (lane == 0) red[warp] = x;
  __syncthreads();
  if (warp == 0) {
    double y = lane < QR_WARPS ? red[lane] : 0.0;
    y = warp_sum(y);
    if (lane == 0) result = y;
  }
  __syncthreads();
  return result;
}

// Warp sums of two values by reduce-scatter: lanes 0-15 finish the first,
// lanes 16-31 the second (5 additions per lane instead of 10).  The result of
// each value is the one a plain xor butterfly leaves in lane 0.
__device__ __forceinline__ void warp_sum2(double& a, double& b, int lane) {
  const bool hi = lane & 16;
  double k = hi ? b : a;
  k += __shfl_xor_sync(0xffffffffu, hi ? a : b, 16);
#pragma unroll
  for (int off = 8; off > 0; off >>= 1) k += __shfl_xor_sync(0xffffffffu, k, off);
  a = __shfl_sync(0xffffffffu, k, 0);
  b = __shfl_sync(0xffffffffu, k, 16);
}

// The same for four values: lanes 0-7, 8-15, 16-23, 24-31 finish a, b, c, d
// (6 additions per lane instead of 20); each result equals warp_sum2's.
__device__ __forceinline__ void warp_sum4(double& a, double& b, double& c, double& d, int lane) {
  const bool hi16 = lane & 16, hi8 = lane & 8;
  double k0 = hi16 ? c : a, k1 = hi16 ? d : b;
  k0 += __shfl_xor_sync(0xffffffffu, hi16 ? a : c, 16);
  k1 += __shfl_xor_sync(0xffffffffu, hi16 ? b : d, 16);
  double k = hi8 ? k1 : k0;
  k += __shfl_xor_sync(0xffffffffu, hi8 ? k0 : k1, 8);
#pragma unroll
  for (int off = 4; off > 0; off >>= 1) k += __shfl_xor_sync(0xffffffffu, k, off);
  a = __shfl_sync(0xffffffffu, k, 0);
  b = __shfl_sync(0xffffffffu, k, 8);
  c = __shfl_sync(0xffffffffu, k, 16);
  d = __shfl_sync(0xffffffffu, k, 24);
}

// Per column, in registers: x = in[0..rows); w = v^H x (one chain over the
// lane's chunks); out = x - v (conj(tau) w) by a fused complex
// multiply-subtract; nu = sum_{i>0} |out_i|^2 (real and imaginary chains).
// R = ceil(rows / 32) chunks per lane; v is zero beyond rows, so only the
// stores are predicated.  The single and the paired form give every column
// the same arithmetic in the same order, so which columns a warp pairs never
// changes a result, and both select paths round alike.
template <int R>
__device__ __forceinline__ void column_update(double2 (&x)[R], const double2* __restrict__ v, double2 s,
                                              double2* __restrict__ out, int rows, int lane, double& nr, double& ni) {
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int i = lane + 32 * u;
    const double2 vi = v[i];
    x[u].x = fma(-vi.x, s.x, x[u].x);
    x[u].x = fma(vi.y, s.y, x[u].x);
    x[u].y = fma(-vi.x, s.y, x[u].y);
    x[u].y = fma(-vi.y, s.x, x[u].y);
    if (i < rows) out[i] = x[u];
    if (u > 0 || lane > 0) {
      nr = fma(x[u].x, x[u].x, nr);
      ni = fma(x[u].y, x[u].y, ni);
    }
  }
}

// A column entry: an L2 load (global columns that other CTAs write) or a
// plain load (columns resident in this CTA's shared memory).
template <bool GLB>
__device__ __forceinline__ double2 ld_entry(const double2* p) {
  if (GLB) return __ldcg(p);
  return *p;
}

template <int R, bool GLB = true>
__device__ __forceinline__ double reflect_column(const double2* __restrict__ in, double2* __restrict__ out,
                                                 const double2* __restrict__ v, double2 ctau, int rows, int lane,
                                                 bool norm) {
  double2 x[R];
  double2 w = make_double2(0.0, 0.0);
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int i = lane + 32 * u;
    x[u] = (i < rows) ? ld_entry<GLB>(in + i) : make_double2(0.0, 0.0);
    w = cfma_conj(v[i], x[u], w);
  }
  warp_sum2(w.x, w.y, lane);
  double nr = 0.0, ni = 0.0;
  column_update<R>(x, v, cmul(ctau, w), out, rows, lane, nr, ni);
  if (!norm) return 0.0;
  double nu = nr + ni;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) nu += __shfl_xor_sync(0xffffffffu, nu, off);
  return __shfl_sync(0xffffffffu, nu, 0);
}

// Two columns at once: independent chains for the FP64 pipe and shared
// reduce-scatter sums.
template <int R, bool GLB = true>
__device__ __forceinline__ void reflect_pair(const double2* __restrict__ in0, double2* __restrict__ out0,
                                             const double2* __restrict__ in1, double2* __restrict__ out1,
                                             const double2* __restrict__ v, double2 ctau, int rows, int lane,
                                             bool norm, double& nu0, double& nu1) {
  double2 x[R], y[R];
  double2 w0 = make_double2(0.0, 0.0), w1 = make_double2(0.0, 0.0);
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int i = lane + 32 * u;
    x[u] = (i < rows) ? ld_entry<GLB>(in0 + i) : make_double2(0.0, 0.0);
    y[u] = (i < rows) ? ld_entry<GLB>(in1 + i) : make_double2(0.0, 0.0);
    const double2 vi = v[i];
    w0 = cfma_conj(vi, x[u], w0);
    w1 = cfma_conj(vi, y[u], w1);
  }
  warp_sum4(w0.x, w0.y, w1.x, w1.y, lane);
  double nr0 = 0.0, ni0 = 0.0, nr1 = 0.0, ni1 = 0.0;
  column_update<R>(x, v, cmul(ctau, w0), out0, rows, lane, nr0, ni0);
  column_update<R>(y, v, cmul(ctau, w1), out1, rows, lane, nr1, ni1);
  nu0 = nr0 + ni0;
  nu1 = nr1 + ni1;
  if (norm) warp_sum2(nu0, nu1, lane);
}

// RMAX: the largest chunk count a kernel instantiation handles (8: l <= 256,
// two CTAs of 128 registers per SM; 16: l <= 512, one CTA per SM).
template <int RMAX, bool GLB = true>
__device__ __forceinline__ double reflect_any(const double2* in, double2* out, const double2* v, double2 ctau,
                                              int rows, int lane, bool norm) {
  switch ((rows + 31) >> 5) {
#define RID_REFLECT_CASE(R) \
    case R: if (R <= RMAX) return reflect_column<(R <= RMAX ? R : 1), GLB>(in, out, v, ctau, rows, lane, norm); break;
    RID_REFLECT_CASE(1) RID_REFLECT_CASE(2) RID_REFLECT_CASE(3) RID_REFLECT_CASE(4)
    RID_REFLECT_CASE(5) RID_REFLECT_CASE(6) RID_REFLECT_CASE(7) RID_REFLECT_CASE(8)
    RID_REFLECT_CASE(9) RID_REFLECT_CASE(10) RID_REFLECT_CASE(11) RID_REFLECT_CASE(12)
    RID_REFLECT_CASE(13) RID_REFLECT_CASE(14) RID_REFLECT_CASE(15) RID_REFLECT_CASE(16)
#undef RID_REFLECT_CASE
    default: break;
  }
  return 0.0;
}

// Pairs only where two columns of registers fit without spilling at two CTAs
// per SM (RMAX = 8, up to 6 chunks); returns false when the caller must take
// the columns one at a time.
#ifndef RID_SEL_PAIR_MAX
#define RID_SEL_PAIR_MAX 6
#endif
template <int RMAX, bool GLB = true>
__device__ __forceinline__ bool reflect_any_pair(const double2* in0, double2* out0, const double2* in1, double2* out1,
                                                 const double2* v, double2 ctau, int rows, int lane, bool norm,
                                                 double& nu0, double& nu1) {
  if (RMAX > 8) return false;
  switch ((rows + 31) >> 5) {
#define RID_PAIR_CASE(R) \
    case R: reflect_pair<(R <= 8 ? R : 1), GLB>(in0, out0, in1, out1, v, ctau, rows, lane, norm, nu0, nu1); return true;
    RID_PAIR_CASE(1) RID_PAIR_CASE(2) RID_PAIR_CASE(3) RID_PAIR_CASE(4) RID_PAIR_CASE(5) RID_PAIR_CASE(6)
#if RID_SEL_PAIR_MAX >= 7
    RID_PAIR_CASE(7)
#endif
#undef RID_PAIR_CASE
    default: return false;
  }
}

constexpr int rid_min_blocks(int rmax) { return rmax <= 8 ? 2 : 1; }

struct SelectArgs {
  double2* Y;
  int64_t ldy;
  int l, k;
  int64_t n;
  int32_t* perm;
  double* part_val;
  int* part_idx;
  unsigned* counter;
  double2* tau;
  int* status;
};

// Post this CTA's best pair; returns true in every thread of the CTA that
// finished last (all other CTAs' writes are then visible to it).
__device__ bool post_and_check_last(const SelectArgs& a, ArgMax best) {
  __shared__ bool am_last;
  __threadfence();
  best = block_argmax(best);
  if (threadIdx.x == 0) {
    a.part_val[blockIdx.x] = best.v;
    a.part_idx[blockIdx.x] = best.i;
    __threadfence();
    const unsigned ticket = atomicAdd(a.counter, 1u);
    am_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

// Run by the last CTA: pick pivot j, swap it into column j, form reflector j.
__device__ void pivot_and_reflect(const SelectArgs& a, int j) {
  __shared__ double2 s_scale;
  ArgMax best{-1.0, INT_MAX};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
    best = better(best, ArgMax{__ldcg(a.part_val + b), __ldcg(a.part_idx + b)});
  best = block_argmax(best);
  if (threadIdx.x == 0) *a.counter = 0u;          // ready for the next launch
  if (!(best.v > 0.0)) {                          // rank(Y) = j < k (Sec. 2)
    if (threadIdx.x == 0) *a.status = RID_ERANK;
    return;
  }
  const int p = best.i;
  double2* colj = a.Y + (int64_t)j * a.ldy;
  if (p != j) {
    double2* colp = a.Y + (int64_t)p * a.ldy;
    for (int i = threadIdx.x; i < a.l; i += blockDim.x) {
      const double2 t = __ldcg(colj + i);
      colj[i] = __ldcg(colp + i);
      colp[i] = t;
    }
    if (threadIdx.x == 0) {
      const int32_t t = a.perm[j];
      a.perm[j] = a.perm[p];
      a.perm[p] = t;
    }
  }
  __syncthreads();
  double part = 0.0;
  for (int i = j + 1 + threadIdx.x; i < a.l; i += blockDim.x) part += cabs2(__ldcg(colj + i));
  const double xnorm2 = block_sum(part);
  if (threadIdx.x < 32) {              // the divisions spread over warp 0 (same bits as one thread)
    double2 tau, scale;
    double beta;
    const bool h = zlarfg_scalars_warp(__ldcg(colj + j), xnorm2, threadIdx.x, tau, scale, beta);
    if (threadIdx.x == 0) {
      if (h) colj[j] = make_double2(beta, 0.0);
      a.tau[j] = tau;
      s_scale = scale;
    }
  }
  __syncthreads();
  const double2 scale = s_scale;
  if (scale.x != 0.0 || scale.y != 0.0)
    for (int i = j + 1 + threadIdx.x; i < a.l; i += blockDim.x) colj[i] = cmul(__ldcg(colj + i), scale);
}

// Step 0 preparation: perm = identity, full column norms, pivot 0.
__global__ void __launch_bounds__(QR_THREADS) select_init_kernel(SelectArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * QR_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * QR_WARPS;
  for (int64_t c = (int64_t)blockIdx.x * QR_THREADS + threadIdx.x; c < a.n;
       c += (int64_t)gridDim.x * QR_THREADS)
    a.perm[c] = (int32_t)c;
  ArgMax best{-1.0, INT_MAX};
  for (int64_t c = gwarp; c < a.n; c += nwarps) {
    const double2* col = a.Y + c * a.ldy;
    double s = 0.0;
    for (int i = lane; i < a.l; i += 32) s += cabs2(col[i]);
    s = warp_sum(s);
    best = better(best, ArgMax{s, (int)c});
  }
  if (post_and_check_last(a, best)) pivot_and_reflect(a, 0);
}

// Step j: apply H_j^H to columns j+1..n-1, new norms, then pivot j+1.
template <int RMAX>
__global__ void __launch_bounds__(QR_THREADS, rid_min_blocks(RMAX)) select_step_kernel(SelectArgs a, int j) {
  __shared__ double2 v[32 * QR_PER_LANE];
  if (*(volatile int*)a.status != RID_OK) return;
  const int lane = threadIdx.x & 31;
  const int rows = a.l - j;                         // rows j..l-1 of the reflector
  const int padded = (rows + 31) & ~31;
  for (int i = threadIdx.x; i < padded; i += blockDim.x)
    v[i] = (i == 0) ? make_double2(1.0, 0.0) : (i < rows ? a.Y[(int64_t)j * a.ldy + j + i] : make_double2(0.0, 0.0));
  const double2 t = a.tau[j];
  const double2 ctau = make_double2(t.x, -t.y);
  __syncthreads();

  const int64_t gwarp = ((int64_t)blockIdx.x * QR_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * QR_WARPS;
  ArgMax best{-1.0, INT_MAX};
  for (int64_t c = j + 1 + gwarp; c < a.n; c += 2 * nwarps) {
    const int64_t c2 = c + nwarps;
    double2* col = a.Y + c * a.ldy + j;
    double nu0 = 0.0, nu1 = 0.0;
    if (c2 < a.n && reflect_any_pair<RMAX>(col, col, a.Y + c2 * a.ldy + j, a.Y + c2 * a.ldy + j, v, ctau, rows,
                                           lane, true, nu0, nu1)) {
      best = better(best, ArgMax{nu0, (int)c});
      best = better(best, ArgMax{nu1, (int)c2});
      continue;
    }
    best = better(best, ArgMax{reflect_any<RMAX>(col, col, v, ctau, rows, lane, true), (int)c});
    if (c2 < a.n) {
      double2* col2 = a.Y + c2 * a.ldy + j;
      best = better(best, ArgMax{reflect_any<RMAX>(col2, col2, v, ctau, rows, lane, true), (int)c2});
    }
  }
  if (j + 1 >= a.k) return;                         // last step: no further pivot
  if (post_and_check_last(a, best)) pivot_and_reflect(a, j + 1);
}

// ---------------------------------------------------------------------------
// All k steps in one cooperative launch (the plan path).
//
// The grid stays resident (a cooperative launch guarantees it) and steps
// through the factorization with one grid barrier per step:
//   - every CTA reduces the posted (norm, position) pairs to the pivot p_j and
//     forms reflector j itself from the winner's posted copy of the column
//     (same data, same code, same block size: bitwise the same result in
//     every CTA, so nothing is broadcast);
//   - warps apply H_j^H to the trailing positions c > j; position p_j takes
//     the column that sat at j (the swap), the pivot's slot is never read, and
//     column j of R is written one step later, once nobody reads slot j;
//   - each CTA posts its best (norm, position) and a copy of that column into
//     the buffer of parity j + 1, so the next step reads posted copies while
//     the slots themselves are rewritten.
// Data written by other CTAs is read with L2 loads (ld.global.cg).  Every
// barrier wait has a clock budget; on expiry the status word becomes
// RID_ETIMEOUT and the CTA returns.
// ---------------------------------------------------------------------------
constexpr long long SEL_WAIT_BUDGET = 4000000000ll;   // clock cycles (~2 s)

struct CoopArgs {
  double2* Y;
  int64_t ldy;
  int l, k;
  int64_t n;
  int32_t* perm;
  double2* tau;
  int* status;
  double2* cand;           // [2][G][l] posted columns
  double* val;             // [2][G] posted norms
  int* idx;                // [2][G] posted positions
  unsigned* bar;           // [0] arrivals, [1] generation
};

// Barrier of `parties` CTAs (the grid) on a.bar: arrivals, then a generation
// count; a CTA that waits longer than `budget` clock cycles sets the status
// word to RID_ETIMEOUT and gets false.
__device__ bool grid_sync(const CoopArgs& a, unsigned parties = 0, long long budget = SEL_WAIT_BUDGET) {
  __shared__ int ok;
  if (parties == 0) parties = gridDim.x;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = a.bar + 1;
    const unsigned g = *gen;
    __threadfence();
    int good = 1;
    if (atomicAdd(a.bar, 1u) == parties - 1) {
      a.bar[0] = 0u;                      // every CTA has arrived: reset, then release
      __threadfence();
      atomicAdd(a.bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (clock64() - t0 > budget) {
          atomicExch(a.status, (int)RID_ETIMEOUT);
          good = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// The CTA's best pair and a copy of that column, into buffer `buf`.
__device__ void post_candidate(const CoopArgs& a, ArgMax best, int buf) {
  const ArgMax r = block_argmax(best);
  const int64_t slot = (int64_t)buf * gridDim.x + blockIdx.x;
  if (r.i != INT_MAX) {
    const double2* col = a.Y + (int64_t)r.i * a.ldy;
    double2* dst = a.cand + slot * a.l;
    for (int i = threadIdx.x; i < a.l; i += QR_THREADS) dst[i] = __ldcg(col + i);
  }
  if (threadIdx.x == 0) {
    a.val[slot] = r.v;
    a.idx[slot] = r.i;
  }
  __threadfence();
}

template <int RMAX>
__global__ void __launch_bounds__(QR_THREADS, rid_min_blocks(RMAX)) select_coop_kernel(CoopArgs a) {
  __shared__ double2 v[32 * QR_PER_LANE];    // reflector j: v[0] = 1, v[i] = row j + i
  __shared__ double2 rc[32 * QR_PER_LANE];   // column j of R with reflector j below it
  __shared__ double2 s_tau, s_scale;
  __shared__ int s_b;
  __shared__ ArgMax s_win;
  const int lane = threadIdx.x & 31;
  const int G = gridDim.x;
  const int l = a.l;
  const int64_t gwarp = ((int64_t)blockIdx.x * QR_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t)G * QR_WARPS;

  // full column norms, the first posting
  for (int64_t c = (int64_t)blockIdx.x * QR_THREADS + threadIdx.x; c < a.n; c += (int64_t)G * QR_THREADS)
    a.perm[c] = (int32_t)c;
  {
    ArgMax best{-1.0, INT_MAX};
    for (int64_t c = gwarp; c < a.n; c += nwarps) {
      const double2* col = a.Y + c * a.ldy;
      double sq = 0.0;
      for (int i = lane; i < l; i += 32) sq += cabs2(__ldcg(col + i));
      sq = warp_sum(sq);
      best = better(best, ArgMax{sq, (int)c});
    }
    post_candidate(a, best, 0);
  }
  if (!grid_sync(a)) return;

  for (int j = 0; j < a.k; ++j) {
    const int buf = j & 1;
    // pivot j: the best posted pair (ties to the lowest position), by warp 0
    if (threadIdx.x < 32) {
      ArgMax w{-1.0, INT_MAX};
      int wb = -1;
      constexpr int PER = 16;            // posted pairs a lane loads before reducing them
      for (int b0 = 0; b0 < G; b0 += 32 * PER) {
        double pv[PER];
        int pi[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          const int b = b0 + lane + 32 * u;
          pv[u] = b < G ? __ldcg(a.val + (int64_t)buf * G + b) : -1.0;
          pi[u] = b < G ? __ldcg(a.idx + (int64_t)buf * G + b) : INT_MAX;
        }
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          const ArgMax nb = better(w, ArgMax{pv[u], pi[u]});
          if (nb.i != w.i) {
            w = nb;
            wb = b0 + lane + 32 * u;
          }
        }
      }
      const ArgMax rw = warp_argmax(w);
      if (wb >= 0 && w.i == rw.i) s_b = wb;
      if (lane == 0) s_win = rw;
    }
    // column j - 1 of R, held since the last step, into its slot
    if (j > 0 && blockIdx.x == (j - 1) % G)
      for (int i = threadIdx.x; i < l; i += QR_THREADS) a.Y[(int64_t)(j - 1) * a.ldy + i] = rc[i];
    __syncthreads();
    const ArgMax r = s_win;
    if (!(r.v > 0.0)) {                                  // rank(Y) = j < k (Sec. 2)
      if (blockIdx.x == 0 && threadIdx.x == 0) *a.status = RID_ERANK;
      return;
    }
    const int p = r.i;
    if (blockIdx.x == 0 && threadIdx.x == 0 && p != j) {
      const int32_t t = a.perm[j];
      a.perm[j] = a.perm[p];
      a.perm[p] = t;
    }
    // reflector j from the posted copy of the pivot column (zlarfg convention)
    const double2* pc = a.cand + ((int64_t)buf * G + s_b) * l;
    for (int i = threadIdx.x; i < l; i += QR_THREADS) rc[i] = __ldcg(pc + i);
    // the norm below the diagonal from the same loads (block_sum's barrier
    // also publishes rc)
    double part = 0.0;
    for (int i = j + 1 + threadIdx.x; i < l; i += QR_THREADS) part += cabs2(__ldcg(pc + i));
    const double xnorm2 = block_sum(part);
    if (threadIdx.x < 32) {
      double2 tau, scale;
      double beta;
      const bool h = zlarfg_scalars_warp(rc[j], xnorm2, lane, tau, scale, beta);
      if (lane == 0) {
        if (h) rc[j] = make_double2(beta, 0.0);
        if (blockIdx.x == 0) a.tau[j] = tau;
        s_tau = tau;
        s_scale = scale;
      }
    }
    __syncthreads();
    const double2 scale = s_scale;
    const bool scaled = scale.x != 0.0 || scale.y != 0.0;
    const int rows = l - j;
    const int padded = (rows + 31) & ~31;
    // v = (1, scaled rows below the diagonal, zero padding); rc keeps the same rows
    for (int i = threadIdx.x; i < padded; i += QR_THREADS) {
      double2 x = make_double2(0.0, 0.0);
      if (i > 0 && i < rows) {
        x = scaled ? cmul(rc[j + i], scale) : rc[j + i];
        rc[j + i] = x;
      }
      v[i] = (i == 0) ? make_double2(1.0, 0.0) : x;
    }
    __syncthreads();

    // H_j^H on positions c > j; position p takes the column that sat at j
    const double2 ctau = make_double2(s_tau.x, -s_tau.y);
    const bool more = j + 1 < a.k;
    ArgMax best{-1.0, INT_MAX};
    // each CTA an even contiguous share of positions j+1 .. n-1; its warps
    // take them in pairs (c, c + QR_WARPS)
    const int64_t first = j + 1, span = a.n - first;
    const int64_t lo = first + span * blockIdx.x / G, hi = first + span * (blockIdx.x + 1) / G;
    const int wid = threadIdx.x >> 5;
    for (int64_t c = lo + wid; c < hi; c += 2 * QR_WARPS) {
      const int64_t c2 = c + QR_WARPS;
      const int64_t src = (c == p) ? j : c, src2 = (c2 == p) ? j : c2;
      const double2* in = a.Y + src * a.ldy;
      double2* out = a.Y + c * a.ldy;
      const double2* in2 = a.Y + src2 * a.ldy;
      double2* out2 = a.Y + c2 * a.ldy;
      if (src != c)
        for (int i = lane; i < j; i += 32) out[i] = __ldcg(in + i);     // the rows above j move along
      if (c2 < hi && src2 != c2)
        for (int i = lane; i < j; i += 32) out2[i] = __ldcg(in2 + i);
      double nu0 = 0.0, nu1 = 0.0;
      if (c2 < hi && reflect_any_pair<RMAX>(in + j, out + j, in2 + j, out2 + j, v, ctau, rows, lane, more, nu0, nu1)) {
        if (more) {
          best = better(best, ArgMax{nu0, (int)c});
          best = better(best, ArgMax{nu1, (int)c2});
        }
        continue;
      }
      nu0 = reflect_any<RMAX>(in + j, out + j, v, ctau, rows, lane, more);
      if (more) best = better(best, ArgMax{nu0, (int)c});
      if (c2 < hi) {
        nu1 = reflect_any<RMAX>(in2 + j, out2 + j, v, ctau, rows, lane, more);
        if (more) best = better(best, ArgMax{nu1, (int)c2});
      }
    }
    if (more) post_candidate(a, best, (j + 1) & 1);
    if (!grid_sync(a)) return;       // after the last step too: slot k-1 may still be read
  }
  // column k - 1 of R
  if (blockIdx.x == (a.k - 1) % G)
    for (int i = threadIdx.x; i < l; i += QR_THREADS) a.Y[(int64_t)(a.k - 1) * a.ldy + i] = rc[i];
}


// ---------------------------------------------------------------------------
// All k steps with Y resident in shared memory (the plan path when the
// columns fit and l <= 256).
//
// One CTA of 512 threads per SM, a cooperative launch.  CTA b owns the
// columns b cpc .. b cpc + cpc - 1 of Y and keeps them in shared memory from
// the first load to the final store: no column crosses L2 between steps.
// Columns never move; the pivoting is bookkept instead.  Every CTA tracks the
// position of each of its columns (ties of the pivot norms still go to the
// lowest position), and all CTAs record the pivot positions p_0 .. p_j and
// the column X_j that sat at position j before swap j (the latest earlier
// step whose pivot position was j left it there, or none did and it is
// column j), so each can apply swap j to its own columns.  At the end every
// column is stored at its final position and perm is written from the
// positions.  The arithmetic of a step is that of the other select paths
// (the same column update, the same order in the pivot's norm, the same
// reflector scalars), so the results agree with them bit for bit.
//
// Exchange: after its update a CTA posts its best (norm, position, column)
// and a copy of that column into the buffer of the next step's parity, then
// raises its flag to the number of steps posted (release).  A step starts
// once every flag has reached it (acquire); a flag wait has a clock budget,
// after which the status word becomes RID_ETIMEOUT and the CTA returns.
// ---------------------------------------------------------------------------
constexpr int RES_THREADS = 512;
constexpr int RES_WARPS = RES_THREADS / 32;
constexpr int RES_MAX_L = 256;
constexpr size_t RES_SMEM_LIMIT = 232448;   // shared memory of one CTA (static + dynamic)

struct ResArgs {
  double2* Y;
  int64_t ldy;
  int l, k;
  int64_t n;
  int32_t* perm;
  double2* tau;
  int* status;
  double2* cand;           // [2][G][l] posted columns
  double* val;             // [2][G] posted norms
  int* pos;                // [2][G] posted positions
  int* col;                // [2][G] posted column indices
  unsigned* flag;          // [G] steps posted by each CTA
  int cpc;                 // columns per CTA
};

struct Best {
  double v;
  int pos;                 // position (the tie key)
  int c;                   // local column
};

__device__ __forceinline__ Best better_res(Best a, Best b) {
  return (b.v > a.v || (b.v == a.v && b.pos < a.pos)) ? b : a;
}

// Block-wide best of 16 warps; result valid in every thread.
__device__ Best block_best(Best a) {
  __shared__ Best red[RES_WARPS];
  __shared__ Best result;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    Best o;
    o.v = __shfl_xor_sync(0xffffffffu, a.v, off);
    o.pos = __shfl_xor_sync(0xffffffffu, a.pos, off);
    o.c = __shfl_xor_sync(0xffffffffu, a.c, off);
    a = better_res(a, o);
  }
  if (lane == 0) red[warp] = a;
  __syncthreads();
  if (warp == 0) {
    Best b = lane < RES_WARPS ? red[lane] : Best{-1.0, INT_MAX, -1};
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      Best o;
      o.v = __shfl_xor_sync(0xffffffffu, b.v, off);
      o.pos = __shfl_xor_sync(0xffffffffu, b.pos, off);
      o.c = __shfl_xor_sync(0xffffffffu, b.c, off);
      b = better_res(b, o);
    }
    if (lane == 0) result = b;
  }
  __syncthreads();
  return result;
}

// Post this CTA's best column for step `step` (buffer step & 1), then raise
// the flag to step + 1.
__device__ void res_post(const ResArgs& a, const double2* cols, int l, Best best, int c_lo, int step) {
  const Best r = block_best(best);
  const int64_t slot = (int64_t)(step & 1) * gridDim.x + blockIdx.x;
  if (r.c >= 0) {
    double2* dst = a.cand + slot * l;
    for (int i = threadIdx.x; i < l; i += RES_THREADS) dst[i] = cols[(int64_t)r.c * l + i];
  }
  if (threadIdx.x == 0) {
    a.val[slot] = r.v;
    a.pos[slot] = r.pos;
    a.col[slot] = r.c >= 0 ? c_lo + r.c : -1;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicExch(a.flag + blockIdx.x, (unsigned)(step + 1));
}

// Wait until every CTA has posted step `step`; false after the clock budget.
// A lane polls its flags (lane, lane + 32, ...) together, one round trip per poll.
constexpr int RES_FLAGS_PER_LANE = 8;                 // grids of up to 256 CTAs
__device__ bool res_wait(const ResArgs& a, int step) {
  __shared__ int ok;
  if (threadIdx.x < 32) {
    const long long t0 = clock64();
    bool good = true;
    unsigned pending = 0;
#pragma unroll
    for (int u = 0; u < RES_FLAGS_PER_LANE; ++u)
      if (threadIdx.x + 32 * u < (int)gridDim.x) pending |= 1u << u;
    while (__any_sync(0xffffffffu, pending != 0)) {
      unsigned f[RES_FLAGS_PER_LANE];
#pragma unroll
      for (int u = 0; u < RES_FLAGS_PER_LANE; ++u)
        if (pending & (1u << u))
          asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(f[u]) : "l"(a.flag + threadIdx.x + 32 * u) : "memory");
#pragma unroll
      for (int u = 0; u < RES_FLAGS_PER_LANE; ++u)
        if ((pending & (1u << u)) && f[u] >= (unsigned)(step + 1)) pending &= ~(1u << u);
      if (pending && clock64() - t0 > SEL_WAIT_BUDGET) {
        atomicExch(a.status, (int)RID_ETIMEOUT);
        good = false;
        pending = 0;
      }
    }
    good = __all_sync(0xffffffffu, good);
    if (threadIdx.x == 0) ok = good;
  }
  __syncthreads();
  return ok != 0;
}

template <int RMAX>
__global__ void __launch_bounds__(RES_THREADS, 1) select_resident_kernel(ResArgs a) {
  extern __shared__ double2 res_cols[];      // cpc columns of l entries, then positions and done marks
  __shared__ double2 v[RES_MAX_L];           // reflector j: v[0] = 1, v[i] = row j + i
  __shared__ double2 rc[RES_MAX_L];          // the pivot column: R above, reflector below
  __shared__ int hp[RES_MAX_L], hx[RES_MAX_L];   // pivot positions and the columns they displaced
  __shared__ double red[QR_WARPS];
  __shared__ double2 s_tau, s_scale;
  __shared__ int s_b, s_x;
  __shared__ ArgMax s_win;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int G = gridDim.x;
  const int l = a.l;
  const int64_t c_lo = (int64_t)blockIdx.x * a.cpc;
  const int64_t c_hi = a.n < c_lo + a.cpc ? a.n : c_lo + a.cpc;
  const int nc = c_hi > c_lo ? (int)(c_hi - c_lo) : 0;
  double2* cols = res_cols;
  int* cpos = (int*)(res_cols + (int64_t)a.cpc * l);
  int* done = cpos + a.cpc;

  // load the CTA's columns; full norms; the first posting
  for (int64_t e = threadIdx.x; e < (int64_t)nc * l; e += RES_THREADS) {
    const int64_t c = e / l, i = e - c * l;
    cols[e] = __ldcg(a.Y + (c_lo + c) * a.ldy + i);
  }
  for (int c = threadIdx.x; c < nc; c += RES_THREADS) {
    cpos[c] = (int)(c_lo + c);
    done[c] = 0;
  }
  __syncthreads();
  {
    Best best{-1.0, INT_MAX, -1};
    for (int c = wid; c < nc; c += RES_WARPS) {
      double sq = 0.0;
      for (int i = lane; i < l; i += 32) sq += cabs2(cols[(int64_t)c * l + i]);
      sq = warp_sum(sq);
      best = better_res(best, Best{sq, cpos[c], c});
    }
    res_post(a, cols, l, best, (int)c_lo, 0);
  }

  int j = 0;
  bool rank_ok = true;
  for (; j < a.k; ++j) {
    if (!res_wait(a, j)) return;
    const int buf = j & 1;
    // pivot j: the best posted pair (ties to the lowest position), by warp 0;
    // warp 1 finds the column at position j before the swap
    if (wid == 0) {
      // the posted pairs of all CTAs, loaded before they are reduced
      ArgMax w{-1.0, INT_MAX};
      int wb = -1;
      double pv[RES_FLAGS_PER_LANE];
      int pp[RES_FLAGS_PER_LANE];
#pragma unroll
      for (int u = 0; u < RES_FLAGS_PER_LANE; ++u) {
        const int b = lane + 32 * u;
        pv[u] = b < G ? __ldcg(a.val + (int64_t)buf * G + b) : -1.0;
        pp[u] = b < G ? __ldcg(a.pos + (int64_t)buf * G + b) : INT_MAX;
      }
#pragma unroll
      for (int u = 0; u < RES_FLAGS_PER_LANE; ++u) {
        const ArgMax nb = better(w, ArgMax{pv[u], pp[u]});
        if (nb.i != w.i) {
          w = nb;
          wb = lane + 32 * u;
        }
      }
      const ArgMax rw = warp_argmax(w);
      if (wb >= 0 && w.i == rw.i) s_b = wb;
      if (lane == 0) s_win = rw;
    } else if (wid == 1) {
      int last = -1;
      for (int jj = lane; jj < j; jj += 32)
        if (hp[jj] == j) last = max(last, jj);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) last = max(last, __shfl_xor_sync(0xffffffffu, last, off));
      if (lane == 0) s_x = last >= 0 ? hx[last] : j;
    }
    __syncthreads();
    const ArgMax r = s_win;
    if (!(r.v > 0.0)) {                                  // rank(Y) = j < k (Sec. 2)
      if (blockIdx.x == 0 && threadIdx.x == 0) *a.status = RID_ERANK;
      rank_ok = false;
      break;
    }
    const int p = r.i;
    const int wbuf = s_b;
    const int q = __ldcg(a.col + (int64_t)buf * G + wbuf);
    const int xj = s_x;
    // reflector j from the posted copy of the pivot column (zlarfg convention);
    // the norm below the diagonal in the order of the 256-thread select CTAs
    const double2* pc = a.cand + ((int64_t)buf * G + wbuf) * l;
    for (int i = threadIdx.x; i < l; i += RES_THREADS) rc[i] = __ldcg(pc + i);
    double part = 0.0;
    if (threadIdx.x < QR_THREADS)
      for (int i = j + 1 + threadIdx.x; i < l; i += QR_THREADS) part += cabs2(__ldcg(pc + i));
    part = warp_sum(part);
    if (lane == 0 && wid < QR_WARPS) red[wid] = part;
    __syncthreads();
    if (wid == 0) {
      double y = lane < QR_WARPS ? red[lane] : 0.0;
      const double xnorm2 = warp_sum(y);
      double2 tau, scale;
      double beta;
      const bool h = zlarfg_scalars_warp(rc[j], xnorm2, lane, tau, scale, beta);
      if (lane == 0) {
        if (h) rc[j] = make_double2(beta, 0.0);
        if (blockIdx.x == 0) a.tau[j] = tau;
        s_tau = tau;
        s_scale = scale;
        hp[j] = p;
        hx[j] = xj;
      }
    }
    __syncthreads();
    const double2 scale = s_scale;
    const bool scaled = scale.x != 0.0 || scale.y != 0.0;
    const int rows = l - j;
    const int padded = (rows + 31) & ~31;
    for (int i = threadIdx.x; i < padded; i += RES_THREADS) {
      double2 x = make_double2(0.0, 0.0);
      if (i > 0 && i < rows) {
        x = scaled ? cmul(rc[j + i], scale) : rc[j + i];
        rc[j + i] = x;
      }
      v[i] = (i == 0) ? make_double2(1.0, 0.0) : x;
    }
    // swap j: the pivot settles at position j, the column from j moves to p
    if (threadIdx.x == 0) {
      if (q >= c_lo && q < c_lo + nc) {
        done[q - c_lo] = 1;
        cpos[q - c_lo] = j;
      }
      if (xj != q && xj >= c_lo && xj < c_lo + nc) cpos[xj - c_lo] = p;
    }
    __syncthreads();
    if (q >= c_lo && q < c_lo + nc)                      // the pivot column: R above, reflector below
      for (int i = j + threadIdx.x; i < l; i += RES_THREADS) cols[(q - c_lo) * (int64_t)l + i] = rc[i];

    // H_j^H on this CTA's remaining columns (rows j..l-1), new norms below row j
    const double2 ctau = make_double2(s_tau.x, -s_tau.y);
    const bool more = j + 1 < a.k;
    Best best{-1.0, INT_MAX, -1};
    for (int c = wid; c < nc; c += 2 * RES_WARPS) {
      const int c2 = c + RES_WARPS;
      const bool l0 = !done[c], l1 = c2 < nc && !done[c2];
      double2* x0 = cols + (int64_t)c * l + j;
      double2* x1 = cols + (int64_t)c2 * l + j;
      double nu0 = 0.0, nu1 = 0.0;
      if (l0 && l1 && reflect_any_pair<RMAX, false>(x0, x0, x1, x1, v, ctau, rows, lane, more, nu0, nu1)) {
        if (more) {
          best = better_res(best, Best{nu0, cpos[c], c});
          best = better_res(best, Best{nu1, cpos[c2], c2});
        }
        continue;
      }
      if (l0) {
        nu0 = reflect_any<RMAX, false>(x0, x0, v, ctau, rows, lane, more);
        if (more) best = better_res(best, Best{nu0, cpos[c], c});
      }
      if (l1) {
        nu1 = reflect_any<RMAX, false>(x1, x1, v, ctau, rows, lane, more);
        if (more) best = better_res(best, Best{nu1, cpos[c2], c2});
      }
    }
    if (more) res_post(a, cols, l, best, (int)c_lo, j + 1);
    __syncthreads();
  }
  (void)rank_ok;
  // every column to its final position (after a rank failure: the state reached)
  for (int64_t e = threadIdx.x; e < (int64_t)nc * l; e += RES_THREADS) {
    const int64_t c = e / l, i = e - c * l;
    a.Y[(int64_t)cpos[c] * a.ldy + i] = cols[e];
  }
  for (int c = threadIdx.x; c < nc; c += RES_THREADS) a.perm[cpos[c]] = (int32_t)(c_lo + c);
}


// |R(0,0)| and the largest column norm of rows k..l-1 over columns k..n-1 of
// a selected Y: one CTA, a warp per column, sums in a fixed order.
__global__ void __launch_bounds__(QR_THREADS) tail_ratio_kernel(const double2* __restrict__ Y, int64_t ldy, int l,
                                                                int k, int64_t n, double* __restrict__ out) {
  __shared__ double red[QR_WARPS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double best = 0.0;
  for (int64_t c = k + wid; c < n; c += QR_WARPS) {
    double sq = 0.0;
    for (int i = k + lane; i < l; i += 32) sq += cabs2(__ldg(Y + c * ldy + i));
    best = fmax(best, warp_sum(sq));
  }
  if (lane == 0) red[wid] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < QR_WARPS; ++w) m = fmax(m, red[w]);
    out[0] = sqrt(cabs2(Y[0]));
    out[1] = sqrt(m);
  }
}
}  // namespace

// CTAs of the cooperative select for n columns (0: use one launch per step).
int rid_select_coop_grid(int device, int num_sms, int64_t n, int l) {
  int coop = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess || !coop) {
    cudaGetLastError();
    return 0;
  }
  const cudaError_t e = l <= 256
      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_coop_kernel<8>, QR_THREADS, 0)
      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_coop_kernel<16>, QR_THREADS, 0);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  int64_t g = (int64_t)per_sm * num_sms;
  const int64_t by_work = (n + 2 * QR_WARPS - 1) / (2 * QR_WARPS);     // at least two columns a warp
  if (g > by_work) g = by_work;
  return (int)(g < 1 ? 1 : g);
}

int rid_select_resident_grid(int device, int num_sms, int64_t n, int l, int* cpc_out, size_t* smem_out) {
  *cpc_out = 0;
  *smem_out = 0;
  if (l < 1 || l > RES_MAX_L || n < 1) return 0;
  int coop = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess || !coop) {
    cudaGetLastError();
    return 0;
  }
  // the attribute is process-wide: always the largest bound, which every shape fits under
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, select_resident_kernel<8>) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const size_t dyn_max = RES_SMEM_LIMIT - fa.sharedSizeBytes - 1024;
  if (cudaFuncSetAttribute(select_resident_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int64_t g = num_sms < 32 * RES_FLAGS_PER_LANE ? num_sms : 32 * RES_FLAGS_PER_LANE;
  const int64_t by_work = (n + 3) / 4;                 // at least four columns a CTA
  if (g > by_work) g = by_work;
  const int64_t cpc = (n + g - 1) / g;
  const size_t smem = (size_t)cpc * l * sizeof(double2) + (size_t)cpc * 2 * sizeof(int);
  if (smem > dyn_max) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_resident_kernel<8>, RES_THREADS, smem) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  g = (n + cpc - 1) / cpc;
  if (g > (int64_t)per_sm * num_sms) return 0;
  *cpc_out = (int)cpc;
  *smem_out = smem;
  return (int)g;
}

cudaError_t rid_launch_tail_ratio(const rid_plan_s* p, const double2* Y, int64_t ldy, double* out) {
  tail_ratio_kernel<<<1, QR_THREADS, 0, p->stream>>>(Y, ldy, p->l, p->k, p->n, out);
  return cudaGetLastError();
}

cudaError_t rid_launch_select(const rid_plan_s* p, double2* Y, int64_t ldy, int32_t* perm) {
  if (p->l > 32 * QR_PER_LANE) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(p->status, 0, sizeof(int), p->stream);
  if (e != cudaSuccess) return e;
  if (p->sel_grid > 0 && p->sel_grid == p->sel_grid_max && p->res_grid > 0) {
    // the default launch shape: Y resident in shared memory
    ResArgs r{Y, ldy, p->l, p->k, p->n, perm, p->tau, p->status, p->res_cand, p->res_val, p->res_pos, p->res_col,
              p->res_flag, p->res_cpc};
    e = cudaMemsetAsync(p->res_flag, 0, (size_t)p->res_grid * sizeof(unsigned), p->stream);
    if (e != cudaSuccess) return e;
    void* args[] = {&r};
    return cudaLaunchCooperativeKernel((const void*)select_resident_kernel<8>, dim3(p->res_grid), dim3(RES_THREADS),
                                       args, p->res_smem, p->stream);
  }
  if (p->sel_grid > 0) {
    CoopArgs c{Y, ldy, p->l, p->k, p->n, perm, p->tau, p->status, p->sel_cand, p->sel_val, p->sel_idx,
               p->sel_bar};
    e = cudaMemsetAsync(p->sel_bar, 0, 2 * sizeof(unsigned), p->stream);
    if (e != cudaSuccess) return e;
    void* args[] = {&c};
    const void* fn = p->l <= 256 ? (const void*)select_coop_kernel<8> : (const void*)select_coop_kernel<16>;
    return cudaLaunchCooperativeKernel(fn, dim3(p->sel_grid), dim3(QR_THREADS), args, 0, p->stream);
  }
  SelectArgs a{Y, ldy, p->l, p->k, p->n, perm, p->qr_val, p->qr_idx, p->qr_counter, p->tau,
               p->status};
  e = cudaMemsetAsync(p->qr_counter, 0, sizeof(unsigned), p->stream);
  if (e != cudaSuccess) return e;
  select_init_kernel<<<p->qr_grid, QR_THREADS, 0, p->stream>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int j = 0; j < p->k; ++j) {
    if (p->l <= 256) select_step_kernel<8><<<p->qr_grid, QR_THREADS, 0, p->stream>>>(a, j);
    else select_step_kernel<16><<<p->qr_grid, QR_THREADS, 0, p->stream>>>(a, j);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Self-test of the bounded waits: an mbarrier that nothing completes (the
// wait every tensor-core kernel uses) and a grid barrier that one CTA more
// than the grid must reach (the select's).  Both must give up after their
// budgets and report RID_ETIMEOUT, and the context stays usable.
// ---------------------------------------------------------------------------
namespace {
__global__ void selftest_wait_kernel(int* status, unsigned* bar) {
  __shared__ uint64_t never;
  if (threadIdx.x == 0) {
    rid_tc::mbar_init(&never, 1);
    rid_tc::fence_barrier_init();
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0 && !rid_tc::mbar_wait(&never, 0, 2000000ll))   // ~1 ms
    atomicExch(status, (int)RID_ETIMEOUT);
  CoopArgs c{};
  c.bar = bar;
  c.status = status + 1;
  grid_sync(c, gridDim.x + 1, 20000000ll);                                           // ~10 ms
}
}  // namespace

extern "C" RID_API rid_status rid_selftest_timeouts(void* stream, int32_t out[2]) {
  if (!out) return RID_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RID_ECUDA;
  char* buf = nullptr;
  if (rid_dev_alloc((void**)&buf, 256, s, dev) != cudaSuccess) return RID_ENOMEM;
  int* status = (int*)buf;
  unsigned* bar = (unsigned*)(buf + 64);
  cudaError_t e = cudaMemsetAsync(buf, 0, 256, s);
  if (e == cudaSuccess) {
    selftest_wait_kernel<<<2, 64, 0, s>>>(status, bar);
    e = cudaGetLastError();
  }
  int h[2] = {-1, -1};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, status, sizeof h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  rid_dev_free(buf, s);
  if (e != cudaSuccess) return RID_ECUDA;
  out[0] = h[0];
  out[1] = h[1];
  return RID_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free pivoted QR.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// allocator's critical section, real-time loops that forbid allocation after
// start-up, or hosts whose device memory is fully owned by a pool they do not
// control.  rid_select_noalloc gives them the select step without a plan:
// its scratch (per-CTA argmax pairs, the last-CTA counter and the reflector
// scalars tau) lives in the fixed-size array below, which every GPU that
// loads this library holds until the process exits.  Every call shares that
// array, so calls whose work overlaps on the GPU (different streams, or
// different host threads on one device) race; calls on one stream are
// ordered and safe.  The array keeps the last call's contents; each call
// clears the counter it relies on before its first launch.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr int NOALLOC_MAX_GRID = 1024;                 // CTAs of one select launch
constexpr int NOALLOC_MAX_STEPS = 32 * QR_PER_LANE;    // reflectors: k <= l <= 512
constexpr size_t NOALLOC_OFF_VAL = 0;
constexpr size_t NOALLOC_OFF_IDX = NOALLOC_OFF_VAL + NOALLOC_MAX_GRID * sizeof(double);
constexpr size_t NOALLOC_OFF_TAU = NOALLOC_OFF_IDX + NOALLOC_MAX_GRID * sizeof(int);
constexpr size_t NOALLOC_OFF_CNT = NOALLOC_OFF_TAU + NOALLOC_MAX_STEPS * sizeof(double2);
constexpr size_t NOALLOC_SCRATCH_BYTES = (NOALLOC_OFF_CNT + sizeof(unsigned) + 255) / 256 * 256;
static_assert(NOALLOC_SCRATCH_BYTES == 20736, "scratch layout changed: update include/rid.h");

static __device__ __align__(256) unsigned char g_select_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_scratch_mutex;
unsigned char* g_scratch_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of g_select_scratch on the current device (looked up once per device).
cudaError_t scratch_address(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_select_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = (unsigned char*)ptr;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" RID_API rid_status rid_select_noalloc(void* Y, int64_t ldy, int32_t l, int64_t n, int32_t k,
                                                 int32_t* perm, int32_t* status, void* stream) {
  if (!Y || !perm || !status) return RID_EINVAL;
  if (l < 1 || n < 1 || k < 1 || k > l || k > n || ldy < l || n > 0x7fffffffLL) return RID_EINVAL;
  if (l > NOALLOC_MAX_STEPS) return RID_EINVAL;        // beyond the static scratch / register tile
  if (((uintptr_t)Y & 15u) || ((uintptr_t)perm & 3u) || ((uintptr_t)status & 3u)) return RID_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return RID_ECUDA;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return RID_ECUDA;
  int64_t grid = (n + 7) / 8;
  if (grid > 4 * (int64_t)sms) grid = 4 * (int64_t)sms;
  if (grid > NOALLOC_MAX_GRID) grid = NOALLOC_MAX_GRID;
  SelectArgs a{(double2*)Y, ldy, l, k, n, perm,
               (double*)(scratch + NOALLOC_OFF_VAL), (int*)(scratch + NOALLOC_OFF_IDX),
               (unsigned*)(scratch + NOALLOC_OFF_CNT), (double2*)(scratch + NOALLOC_OFF_TAU),
               (int*)status};
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return RID_ECUDA;
  select_init_kernel<<<(unsigned)grid, QR_THREADS, 0, s>>>(a);
  if (cudaGetLastError() != cudaSuccess) return RID_ECUDA;
  for (int j = 0; j < k; ++j) {
    if (l <= 256) select_step_kernel<8><<<(unsigned)grid, QR_THREADS, 0, s>>>(a, j);
    else select_step_kernel<16><<<(unsigned)grid, QR_THREADS, 0, s>>>(a, j);
    if (cudaGetLastError() != cudaSuccess) return RID_ECUDA;
  }
  return RID_OK;
}
