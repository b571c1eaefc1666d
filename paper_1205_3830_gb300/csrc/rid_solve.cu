// Factorization of R (Sec. 2, "R2 = R1 T"): T = R1^-1 R2 by back substitution.
//
// The right-hand sides are independent (Sec. 3.2: the paper gives each
// processor its own column), so each CTA takes a block of NR columns of R2
// into shared memory and eliminates from the last row up: row j of the block
// is divided by R1_jj, then column j of R1 (rows 0..j, staged in shared
// memory) updates every row above it.  Column j - 1 is loaded while column j
// updates (two staging buffers), so the L2 latency stays off the chain.  R1
// (k x k, at most a few hundred KB) stays in L2 for all CTAs.
#include <climits>
#include <cstdint>

#include "rid_internal.cuh"

namespace {

constexpr int SOLVE_THREADS = 256;
constexpr size_t SOLVE_SMEM_BUDGET = 200 * 1024;
constexpr size_t SOLVE_SMEM_LIMIT = 227 * 1024;    // shared memory of an SM available to CTAs

__global__ void __launch_bounds__(SOLVE_THREADS)
solve_kernel(const double2* __restrict__ Y, int64_t ldy, int k, int64_t n, int nr,
             double2* __restrict__ T, int64_t ldt) {
  extern __shared__ double2 smem[];
  double2* rhs = smem;                  // k x nr, row i at rhs[i * nr]
  double2* rcol = smem + (size_t)k * nr; // [2][k]: column j of R1, rows 0..j, by the parity of j
  const int tid = threadIdx.x;
  const int64_t c0 = (int64_t)blockIdx.x * nr;      // first column of T in this block
  const int64_t ncols = n - k;
  int nvalid = (int)((ncols - c0) < nr ? (ncols - c0) : nr);

  for (int e = tid; e < k * nr; e += SOLVE_THREADS) {
    const int c = e / k, i = e - c * k;
    rhs[i * nr + c] = (c < nvalid) ? Y[i + (k + c0 + c) * ldy] : make_double2(0.0, 0.0);
  }
  for (int i = tid; i < k; i += SOLVE_THREADS) rcol[((k - 1) & 1) * k + i] = Y[i + (int64_t)(k - 1) * ldy];
  for (int j = k - 1; j >= 0; --j) {
    const double2* rc = rcol + (j & 1) * k;
    // column j - 1 (rows 0..j-1; k <= 2 SOLVE_THREADS) into registers now, into its buffer after the update
    double2 pre[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = tid + q * SOLVE_THREADS;
      if (i < j) pre[q] = Y[i + (int64_t)(j - 1) * ldy];
    }
    __syncthreads();
    if (tid < nr) rhs[j * nr + tid] = cdiv(rhs[j * nr + tid], rc[j]);
    __syncthreads();
    for (int e = tid; e < j * nr; e += SOLVE_THREADS) {
      const int i = e / nr, c = e - i * nr;
      const double2 r = rc[i], t = rhs[j * nr + c];
      double2 x = rhs[e];
      x.x = fma(-r.x, t.x, x.x);
      x.x = fma(r.y, t.y, x.x);
      x.y = fma(-r.x, t.y, x.y);
      x.y = fma(-r.y, t.x, x.y);
      rhs[e] = x;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = tid + q * SOLVE_THREADS;
      if (i < j) rcol[((j - 1) & 1) * k + i] = pre[q];
    }
  }
  __syncthreads();
  for (int e = tid; e < k * nr; e += SOLVE_THREADS) {
    const int c = e / k, i = e - c * k;
    if (c < nvalid) T[i + (c0 + c) * ldt] = rhs[i * nr + c];
  }
}

}  // namespace

size_t rid_solve_smem_bytes(int k, int* nr_out) {
  int nr = 32;
  while (nr > 1 && (size_t)(k * nr + 2 * k) * sizeof(double2) > SOLVE_SMEM_BUDGET) nr >>= 1;
  if (nr_out) *nr_out = nr;
  if (k > 2 * SOLVE_THREADS) return SIZE_MAX;     // the kernel stages two rows of a column per thread
  return (size_t)(k * nr + 2 * k) * sizeof(double2);
}

namespace {

// Right-hand sides per CTA: the FP64 pipe of an SM is shared by its CTAs, so
// the time is set by the busiest SM, ceil(CTAs / SMs) blocks of nr columns.
// Among widths that fit (and keep a step's update worth a barrier, nr >= 8),
// take the one that minimizes that product.
int solve_block_width(int k, int64_t ncols, int sms, int nr_max) {
  int best = nr_max;
  int64_t best_cost = INT64_MAX;
  for (int nr = nr_max; nr >= 8 || (nr >= 1 && nr == nr_max); --nr) {
    const size_t smem = (size_t)(k * nr + 2 * k) * sizeof(double2);
    int per_sm = (int)((size_t)(SOLVE_SMEM_LIMIT) / smem);
    if (per_sm > 2048 / SOLVE_THREADS) per_sm = 2048 / SOLVE_THREADS;
    if (per_sm < 1) continue;
    const int64_t ctas = (ncols + nr - 1) / nr;
    const int64_t waves = (ctas + (int64_t)sms * per_sm - 1) / ((int64_t)sms * per_sm);
    const int64_t cost = ((ctas + sms - 1) / sms) * nr + waves;   // busiest SM's columns (+ a wave tie-break)
    if (cost < best_cost) {
      best_cost = cost;
      best = nr;
    }
  }
  return best;
}

}  // namespace

cudaError_t rid_launch_solve(const rid_plan_s* p, const double2* Y, int64_t ldy, double2* T,
                             int64_t ldt) {
  const int64_t ncols = p->n - p->k;
  if (ncols <= 0) return cudaSuccess;
  int nr_max = 0;
  if (rid_solve_smem_bytes(p->k, &nr_max) > SOLVE_SMEM_BUDGET) return cudaErrorInvalidValue;
  const int nr = solve_block_width(p->k, ncols, p->num_sms, nr_max);
  const size_t smem = (size_t)(p->k * nr + 2 * p->k) * sizeof(double2);
  // one fixed limit for every plan: the attribute is process-wide, and plans
  // on other host threads launch this kernel concurrently
  cudaError_t e = cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SOLVE_SMEM_BUDGET);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((ncols + nr - 1) / nr);
  solve_kernel<<<blocks, SOLVE_THREADS, smem, p->stream>>>(Y, ldy, p->k, p->n, nr, T, ldt);
  return cudaGetLastError();
}
